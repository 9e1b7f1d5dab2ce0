"""kg_overlaps_noalloc: the overlap entry point for callers that cannot
allocate device memory at call time (for example code under a fixed
device-memory budget, or with a memory pool that must not grow).  It must
give the same results as kg_overlaps, call after call, although every call
reuses the same fixed scratch arrays.  This file is collected last on
purpose, so that a run stopping at the first failure has run everything else."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1109_1205_gb300 as kg  # noqa: E402


def _noalloc(X, n_x, Y, n_y, d, G, stream):
    fn = kg.lib.kg_overlaps_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong,
                   ctypes.c_void_p, ctypes.c_void_p]
    return fn(X.data_ptr(), n_x, Y.data_ptr(), n_y, d, G.data_ptr(), stream.cuda_stream)


def _case(seed, n_x, n_y, d):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n_x, d)) + 1j * rng.standard_normal((n_x, d))
    Y = rng.standard_normal((n_y, d)) + 1j * rng.standard_normal((n_y, d))
    return torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()


def test_noalloc_matches_allocating_entry_point_twice():
    st = torch.cuda.current_stream()
    for seed, (n_x, n_y, d) in enumerate([(12, 12, 731808), (5, 64, 20001)]):
        X, Y = _case(seed, n_x, n_y, d)
        ref = torch.empty((n_y, n_x), dtype=torch.complex128, device="cuda")
        kg.kg_overlaps(X, n_x, Y, n_y, d, ref, st)
        for _ in range(2):  # two calls in a row share the fixed scratch
            G = torch.full((n_y, n_x), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
            assert _noalloc(X, n_x, Y, n_y, d, G, st) == kg.KG_OK, kg.kg_last_error()
            torch.cuda.synchronize()
            scale = max(1.0, float(np.sqrt(d)))
            assert torch.max(torch.abs(G - ref)).item() < 1e-12 * scale


def test_noalloc_rejects_sizes_beyond_its_scratch():
    st = torch.cuda.current_stream()
    X, Y = _case(7, 2, 65, 64)
    G = torch.empty((65, 2), dtype=torch.complex128, device="cuda")
    rc = _noalloc(X, 2, Y, 65, 64, G, st)
    assert rc == kg.KG_EINVAL
    assert "limit of 64 columns" in kg.kg_last_error()
