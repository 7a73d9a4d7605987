"""The allocation-free entry point against the oracle and the handle-based solver.

fd_forward_noalloc serves callers that cannot allocate device memory (a
framework's caching allocator owns the device; a serving loop must not pay the
device-wide synchronisation of cudaMalloc/cudaFree). It runs the expanded-form
step on buffers the caller owns and keeps its scratch in a static device array.
This test checks two calls in a row (the second resuming where the first
stopped) against the FP64 oracle and against fd_forward of a handle with the
same inputs, within the parity tolerance, and that the reported max |u|
covers the wavefield. The file
name sorts last so that a run stopping at the first failure has already run
every other test.
"""
import numpy as np
import pytest

import paper_1912_00695_gb300 as fd
from paper_1912_00695_gb300 import _abi, inputs
from harness import rel_l2, run_oracle

pytestmark = pytest.mark.gpu

TOL = 1e-5


def test_noalloc_matches_oracle_and_handle_on_two_calls(oracle_mod):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(21)
    interior, nbl, k = (37, 45, 51), 6, 8
    vel = inputs.smooth_random_velocity(interior, nbl, rng, sigma=4.0)
    spec = inputs.ShotSpec(interior, nbl, k, vel, (1, 43, 25), 25.0, 60)
    shape = spec.shape
    m = spec.m
    eta = oracle_mod.default_damping(m, nbl, inputs.H).astype(np.float32)
    dt = 0.9 * oracle_mod.dt_max(k, inputs.H, spec.vmax)
    interior_nodes = [(1, 43, 25), (20, 10, 40)]
    wavelets = [inputs.ricker(25.0, dt, 60), inputs.ricker(18.0, dt, 45, amplitude=2.0)]
    n1, n2 = 23, 30

    # handle-based reference, same stencil form
    shot = fd.Shot(interior, k, inputs.H, dt, nbl, form="expanded", kernel="stream")
    shot.set_model(m, eta)
    for node, w in zip(interior_nodes, wavelets):
        shot.inject(*node, w)
    shot.forward(n1)
    ref1 = shot.wavefield(0)
    shot.forward(n2)
    ref2 = shot.wavefield(0)
    shot.close()
    srcs = list(zip(interior_nodes, wavelets))
    want1, want1_prev = run_oracle(oracle_mod, spec, n1, dt, eta, sources=srcs)
    want2, _ = run_oracle(oracle_mod, spec, n2, dt, eta, sources=srcs, state=(want1, want1_prev, n1))

    dev = torch.device("cuda", 0)
    u = torch.zeros(shape, dtype=torch.float32, device=dev)
    u_prev = torch.zeros(shape, dtype=torch.float32, device=dev)
    d_m = torch.from_numpy(m).to(dev)
    d_eta = torch.from_numpy(eta).to(dev)
    ld = max(len(w) for w in wavelets)
    wav = np.zeros((len(wavelets), ld), dtype=np.float32)
    for i, w in enumerate(wavelets):
        wav[i, :len(w)] = w
    d_wav = torch.from_numpy(wav).to(dev)
    nodes = [tuple(c + nbl for c in n) for n in interior_nodes]
    stream = torch.cuda.current_stream().cuda_stream

    # call 1: steps 0..n1-1 from zero fields
    amax1 = _abi.fd_forward_noalloc(u, u_prev, d_m, d_eta, shape, k, inputs.H, dt, nodes, d_wav,
                                    ld, step0=0, nt=n1, stream=stream)
    newest, older = (u, u_prev) if n1 % 2 == 0 else (u_prev, u)
    got1 = newest.cpu().numpy()
    assert rel_l2(got1, want1) <= TOL
    assert rel_l2(got1, ref1) <= TOL
    assert np.isfinite(amax1) and amax1 >= np.abs(got1).max() > 0

    # call 2: resume at step n1 with the levels the first call left
    amax2 = _abi.fd_forward_noalloc(newest, older, d_m, d_eta, shape, k, inputs.H, dt, nodes, d_wav,
                                    ld, step0=n1, nt=n2, stream=stream)
    newest2 = newest if n2 % 2 == 0 else older
    got2 = newest2.cpu().numpy()
    assert rel_l2(got2, want2) <= TOL
    assert rel_l2(got2, ref2) <= TOL
    assert np.isfinite(amax2) and amax2 >= np.abs(got2).max() > 0


def test_noalloc_rejects_sizes_beyond_scratch():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    tiny = torch.zeros(8, dtype=torch.float32, device=dev)
    # Ny * Nz = 4200 * 4200 needs more than 16384 CTAs per step; rejected before any launch
    with pytest.raises(fd.FdError) as e:
        _abi.fd_forward_noalloc(tiny, tiny, tiny, None, (16, 4200, 4200), 8, 10.0, 1e-3, nt=1)
    assert e.value.code == fd.FD_EINVAL
    assert "16384" in fd.fd_last_error()
