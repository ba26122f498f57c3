"""The allocation-free step entry point (ms_step_csr_noalloc) against the
regular one (ms_create + ms_step + ms_get_state).

Callers that cannot allocate device memory -- code running under CUDA graph
capture, plugins whose host framework owns all device memory, real-time
loops -- pass all inputs and outputs themselves; the working memory is a
fixed array inside the library.  This file is collected last so that a run
stopping at its first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ms():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2207_09334_gb300 as ms
    ms.load()
    return ms


def csr(system):
    """Both-direction CSR incidence of the system's springs (host arrays)."""
    ij = system["ij"]; N = system["x"].shape[0]
    a = np.concatenate([ij[:, 0], ij[:, 1]]); b = np.concatenate([ij[:, 1], ij[:, 0]])
    e = np.concatenate([np.arange(len(ij))] * 2)
    order = np.lexsort((b, a))
    a, b, e = a[order], b[order], e[order]
    row = np.zeros(N + 1, np.int32)
    np.add.at(row, a + 1, 1)
    row = np.cumsum(row).astype(np.int32)
    c = np.broadcast_to(np.asarray(system["c"], np.float32), (len(ij),))
    return row, b.astype(np.int32), system["k"][e].astype(np.float32), c[e].astype(np.float32), \
        system["L0"][e].astype(np.float32)


def step_noalloc(ms, system, params, nsteps, x_in, v_in):
    import torch
    lib = ms.load()
    p = ms.make_params(params)
    N = system["x"].shape[0]
    row, partner, k, c, L0 = csr(system)
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    dm, dfix = d(system["m"].astype(np.float32)), d(system["fixed"].astype(np.uint8))
    drow, dp, dk, dc, dL = d(row), d(partner), d(k), d(c), d(L0)
    xo = torch.empty((N, 3), device="cuda"); vo = torch.empty((N, 3), device="cuda")
    ptr = lambda t: C.c_void_p(t.data_ptr())
    rc = lib.ms_step_csr_noalloc(C.byref(p), N, ptr(x_in), ptr(v_in), ptr(dm), ptr(dfix), ptr(drow), ptr(dp),
                                 ptr(dk), ptr(dc), ptr(dL), int(nsteps), ptr(xo), ptr(vo),
                                 C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.ms_last_error().decode()
    torch.cuda.synchronize()
    return xo, vo


def test_noalloc_matches_regular_step_on_two_calls_in_a_row(ms):
    import torch
    s = synth.soft_cube(n=8, z0=0.001)
    s["v"][:] = np.array([0.2, -0.1, -0.5], np.float32)
    p = synth.soft_cube_params(contact=True)
    size = float(np.ptp(s["x"], axis=0).max())
    with ms.Sim(s, p, kernel="gather") as sim:
        sim.step(150)
        x1, v1 = sim.get_state()
        sim.step(150)
        x2, v2 = sim.get_state()
    x0 = torch.tensor(s["x"], device="cuda"); v0 = torch.tensor(s["v"], device="cuda")
    xa, va = step_noalloc(ms, s, p, 150, x0, v0)          # first call
    xb, vb = step_noalloc(ms, s, p, 150, xa.clone(), va.clone())   # second call, continuing
    for got, want in ((xa, x1), (xb, x2)):
        err = np.abs(got.cpu().numpy() - want).max()
        assert err <= 1e-4 * size, (err, size)
    assert np.abs(vb.cpu().numpy() - v2).max() <= 1e-2 * np.abs(v2).max()


def test_noalloc_rejects_systems_beyond_its_scratch(ms):
    import torch
    lib = ms.load()
    p = ms.make_params(synth.params())
    N = 262144 + 1
    t = torch.zeros(8, device="cuda")
    ptr = C.c_void_p(t.data_ptr())
    rc = lib.ms_step_csr_noalloc(C.byref(p), N, ptr, ptr, ptr, None, ptr, ptr, ptr, ptr, ptr, 1, ptr, ptr, None)
    assert rc == 1 and "262144" in lib.ms_last_error().decode()
