"""teuk_substep_noalloc: Lax-Wendroff iterations that allocate no device memory.

It is meant for callers whose device memory is owned by a pool of their own, or who cannot
afford cudaMalloc / cudaFree in their stepping loop. The test drives it through the C ABI
with caller-owned device buffers, twice in a row (out of place, then in place), on both
multi-word arithmetic engines, and checks the result against teuk_substep on the same data
and against the 256-bit CPU oracle, within the parity tolerances of the GPU tests. It also
checks that sizes beyond the fixed scratch array and misaligned buffers are refused."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1006_0663_gb300 import teuk

pytestmark = pytest.mark.gpu

TOL = {1: 1e-12, 2: 1e-26, 4: 1e-55}


def _torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _word_rel_err(got, want):
    diff = 0.0
    for k in reversed(range(want.shape[1])):
        diff = diff + (got[:, k] - want[:, k])
    return np.abs(diff).max() / np.abs(want[:, 0]).max()


P_SMALL = dict(M=1.0, a=0.9, s=-2, m=2, rstar_min=-30.0, rstar_max=50.0, n_r=41, n_theta=24,
               substeps=4)


@pytest.mark.parametrize("W,engine", [(1, 0), (2, 0), (2, 1), (4, 0), (4, 1)])
def test_noalloc_matches_substep_two_calls(W, engine):
    torch = _torch_cuda()
    p = P_SMALL
    g = teuk.Teuk(precision=W, **p)
    if engine:
        g.set_engine(engine)
    g.set_initial_pulse(12.0, 4.0, 0.8, 0.55, 2)
    u0 = g.get_state()
    pitch = (p["n_theta"] + 15) // 16 * 16
    buf_in = torch.zeros((4, W, p["n_r"], pitch), dtype=torch.float64, device="cuda")
    buf_out = torch.full((4, W, p["n_r"], pitch), 7.0, dtype=torch.float64, device="cuda")
    buf_in[..., : p["n_theta"]] = torch.from_numpy(u0).cuda()
    torch.cuda.synchronize()
    L = teuk.lib()
    rc = L.teuk_substep_noalloc(g._h, ctypes.c_void_p(buf_in.data_ptr()),
                                ctypes.c_void_p(buf_out.data_ptr()), 3)
    assert rc == 0, L.teuk_last_error(g._h)
    rc = L.teuk_substep_noalloc(g._h, ctypes.c_void_p(buf_out.data_ptr()),
                                ctypes.c_void_p(buf_out.data_ptr()), 3)
    assert rc == 0, L.teuk_last_error(g._h)
    g.sync()
    torch.cuda.synchronize()
    got = buf_out[..., : p["n_theta"]].cpu().numpy()
    g.substep(6)  # the existing entry point on the same initial data
    want = g.get_state()
    assert np.abs(want[:, 0]).max() > 0.05
    assert _word_rel_err(got, want) < TOL[W]
    assert np.all(got[:, :, 0] == 0) and np.all(got[:, :, -1] == 0)
    # and against the oracle: the same six iterations in 256-bit arithmetic
    o = oracle.Oracle(M=p["M"], a=p["a"], s=p["s"], m=p["m"], rstar_min=p["rstar_min"],
                      rstar_max=p["rstar_max"], n_r=p["n_r"], n_theta=p["n_theta"], dt=0.0,
                      substeps=p["substeps"], bits=256)
    o.pulse(12.0, 4.0, 0.8, 0.55, 2)
    o.step(6)
    err, umax = o.max_rel_err(got)
    assert umax > 0.05 and err < TOL[W], err


def test_noalloc_rejects_misaligned_buffers():
    torch = _torch_cuda()
    p = P_SMALL
    g = teuk.Teuk(precision=2, **p)
    g.set_engine(1)
    pitch = (p["n_theta"] + 15) // 16 * 16
    n = 4 * 2 * p["n_r"] * pitch
    buf = torch.zeros(n + 2, dtype=torch.float64, device="cuda")
    L = teuk.lib()
    base = buf.data_ptr()
    for u_in, u_out in ((base + 8, base), (base, base + 8)):
        rc = L.teuk_substep_noalloc(g._h, ctypes.c_void_p(u_in), ctypes.c_void_p(u_out), 1)
        assert rc == teuk.ERR_INVALID_ARG
        assert b"16-byte" in L.teuk_last_error(g._h)
    g.sync()  # nothing was launched: the handle is still usable


def test_noalloc_rejects_sizes_beyond_the_fixed_array():
    torch = _torch_cuda()
    # 4 * 1 word * 8199 rows * 64 = 2,098,944 doubles > 2^21
    g = teuk.Teuk(precision=1, M=1.0, a=0.5, s=0, m=0, rstar_min=-50.0, rstar_max=150.0,
                  n_r=8200, n_theta=64, substeps=1)
    buf = torch.zeros((4, 1, 8200, 64), dtype=torch.float64, device="cuda")
    L = teuk.lib()
    rc = L.teuk_substep_noalloc(g._h, ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(buf.data_ptr()), 1)
    assert rc == teuk.ERR_INVALID_ARG
    assert b"2^21" in L.teuk_last_error(g._h)
