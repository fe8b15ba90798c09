"""The allocation-free entry point mbmd_objective_noalloc, for callers that
cannot allocate device memory (a framework's own allocator owns the device
memory, a fixed memory budget, or loops that must not call cudaMalloc /
cudaFree).  Called through the C ABI and checked against the allocating
mbmd_objective on the same inputs, twice in a row (the static scratch keeps
the previous call's contents, which must not leak into the next result).

Kept in its own file so that it is collected last."""
import ctypes

import numpy as np
import pytest

import synth
from _helpers import to_dev

pytestmark = pytest.mark.gpu


def _call_noalloc(lib, Q, S, l, y, out, stream):
    dp = ctypes.POINTER(ctypes.c_double)
    Qc = np.ascontiguousarray(Q, dtype=np.float64)
    Sc = np.ascontiguousarray(S, dtype=np.float64)
    return lib.mbmd_objective_noalloc(Q.shape[1], Q.shape[0], S.shape[0], Qc.ctypes.data_as(dp),
                                      Sc.ctypes.data_as(dp), ctypes.c_void_p(l.data_ptr()),
                                      ctypes.c_void_p(y.data_ptr()), y.shape[1], ctypes.c_void_p(out.data_ptr()),
                                      stream)


def test_noalloc_objective_matches_allocating_entry_point():
    import torch

    import paper_2010_01371_gb300 as p
    lib = p.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = []
    prob = synth.config3(n_views=12, n_u=301)                      # 2 materials, 121 energies, 2 channels
    cases.append((prob.Q, prob.S, 0.9 * prob.truth, prob.y))
    rng = np.random.default_rng(3)
    l1 = rng.uniform(0.0, 4.0, (1, 70001))                          # standard CT, 1x1x1, ragged length
    y1 = rng.poisson(1e4 * np.exp(-l1)).astype(float)
    cases.append((np.ones((1, 1)), np.full((1, 1), 1e4), 1.02 * l1, y1))
    for Q, S, l, y in cases:
        spec = p.Spectrum(Q, S)
        ld, yd = to_dev(l), to_dev(y)
        want = float(p.mbmd_objective(None, spec, ld, yd).item())
        for _ in range(2):                                          # two calls in a row
            out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            st = _call_noalloc(lib, Q, S, ld, yd, out, stream)
            assert st == 0, lib.mbir_last_error()
            torch.cuda.synchronize()
            got = float(out.item())
            assert abs(got - want) <= 1e-5 * abs(want), (got, want)


def test_noalloc_rejects_sizes_beyond_the_scratch():
    import torch

    import paper_2010_01371_gb300 as p
    lib = p.lib()
    Q = np.ones((257, 1))
    S = np.ones((1, 257))
    l = torch.zeros((1, 4), device="cuda")
    y = torch.ones((1, 4), device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = _call_noalloc(lib, Q, S, l, y, out, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == -1
    assert b"static scratch" in lib.mbir_last_error()


def test_noalloc_rejects_a_capturing_stream():
    """The call stages its table with a pageable host copy, which a CUDA graph
    would replay from a stack buffer that no longer exists; made on a stream
    that is capturing, it returns MBIR_ERR_ARG and enqueues nothing."""
    import torch

    import paper_2010_01371_gb300 as p
    lib = p.lib()
    Q, S = np.ones((1, 1)), np.full((1, 1), 1e4)
    l = torch.zeros((1, 8), device="cuda")
    y = torch.ones((1, 8), device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=side):
        out.fill_(1.0)
        st = _call_noalloc(lib, Q, S, l, y, out, ctypes.c_void_p(side.cuda_stream))
    assert st == -1
    assert b"capturing" in lib.mbir_last_error()
    g.replay()
    torch.cuda.synchronize()
    assert float(out.item()) == 1.0
