"""CPU checks of the C ABI: the library builds, loads and exports every entry
point include/parquet.h declares; argument validation needs no GPU."""
import ctypes as C
import os
import re

import pytest

from paper_1510_03330_gb300 import binding
from paper_1510_03330_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return binding.load_library()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "parquet.h")).read()
    return sorted(set(re.findall(r"PQ_API[^;(]*?\b(pq_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n


def test_default_options(lib):
    o = binding.default_options()
    assert o.precision == 0 and o.mix_alpha == 0.5 and o.sigma2_box_factor == 3
    assert o.hop == 1.0 and o.tau_panels == 64 and o.tau_order == 16 and o.tau_matsubara == 2048
    assert not o.dev_alloc and not o.dev_free


@pytest.mark.parametrize("args,msg", [
    ((5, 1.0, 1.0, 0.0, 1, 8, 7), "unknown lattice"),
    ((1, -1.0, 1.0, 0.0, 2, 8, 7), "beta"),
    ((0, 1.0, 1.0, 0.0, 2, 8, 7), "L must be"),
    ((1, 1.0, 1.0, 0.0, 2, 7, 7), "n_nu"),
    ((1, 1.0, 1.0, 0.0, 2, 8, 0), "n_Omega"),
    ((1, 1.0, 1.0, 0.0, 2, 200, 200), "too large"),
])
def test_init_rejects_bad_arguments_without_touching_the_gpu(lib, args, msg):
    h = C.c_void_p()
    st = lib.pq_init(C.byref(h), *args, None)
    assert st == binding.PQ_EINVAL
    assert msg in lib.pq_last_error(None).decode()
    assert not h.value


def test_bad_options_are_rejected(lib):
    o = binding.default_options()
    o.mix_alpha = 0.0
    h = C.c_void_p()
    assert lib.pq_init(C.byref(h), 1, 2.0, 1.0, 0.0, 2, 8, 7, C.byref(o)) == binding.PQ_EINVAL
    o = binding.default_options()
    o.precision = 9
    assert lib.pq_init(C.byref(h), 1, 2.0, 1.0, 0.0, 2, 8, 7, C.byref(o)) == binding.PQ_EINVAL


def test_null_context_calls_are_safe(lib):
    assert lib.pq_iterate(None, 1, 0.0, None, None) == binding.PQ_EINVAL
    lib.pq_destroy(None)
    assert lib.pq_step_name(0) == b"dyson"


def test_bad_q_chunk_is_rejected(lib):
    o = binding.default_options()
    o.q_chunk = -1
    h = C.c_void_p()
    assert lib.pq_init(C.byref(h), 1, 2.0, 1.0, 0.0, 2, 8, 7, C.byref(o)) == binding.PQ_EINVAL
    assert "q_chunk" in lib.pq_last_error(None).decode()


@pytest.mark.parametrize("field,value,word", [("assembly", 2, "assembly"), ("kernel_level", 3, "kernel_level"),
                                              ("edge_rule", 2, "edge_rule"), ("sde", 2, "sde")])
def test_bad_kernel_options_are_rejected(lib, field, value, word):
    o = binding.default_options()
    assert (o.assembly, o.kernel_level, o.edge_rule, o.sde) == (0, 0, 0, 0)
    setattr(o, field, value)
    h = C.c_void_p()
    assert lib.pq_init(C.byref(h), 1, 2.0, 1.0, 0.0, 2, 8, 7, C.byref(o)) == binding.PQ_EINVAL
    assert word in lib.pq_last_error(None).decode()


def test_batch_arguments_are_checked_without_touching_the_gpu(lib):
    o = binding.BatchOptions()
    lib.pq_batch_default_options(C.byref(o))
    assert (o.tile_cols, o.order, o.time_steps) == (0, -1, 0)
    h = C.c_void_p()
    assert lib.pq_batch_create(C.byref(h), None, 0, None) == binding.PQ_EINVAL
    assert not h.value
    arr = (C.c_void_p * 1)(None)
    assert lib.pq_batch_create(C.byref(h), arr, 1, None) == binding.PQ_EINVAL
    assert "NULL" in lib.pq_last_error(None).decode()
    o.tile_cols = 96
    assert lib.pq_batch_create(C.byref(h), arr, 1, C.byref(o)) == binding.PQ_EINVAL
    assert "tile_cols" in lib.pq_last_error(None).decode()
    assert lib.pq_batch_iterate(None, 1, None) == binding.PQ_EINVAL
    lib.pq_batch_destroy(None)


def test_set_lambda_without_context_is_rejected(lib):
    assert lib.pq_set_Lambda(None, 0, None, 2) == binding.PQ_EINVAL
