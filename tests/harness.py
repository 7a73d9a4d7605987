"""Test-side helpers: run the same seeded shot through the C-ABI and the oracle.

Both sides receive identical inputs from paper_1912_00695_gb300.inputs (the
model m as float32, the wavelet as float32 samples) and the same dt and damping
eta. dt and the default eta come from the oracle (its stability limit and its
damping profile, eta rounded to float32), so no value the oracle consumes
originates in the library; the library's own helpers are checked against these
in tests/test_abi_cpu.py.
"""
from __future__ import annotations

import numpy as np

import paper_1912_00695_gb300 as fd
from paper_1912_00695_gb300 import inputs


def dt_for(spec, frac=0.9) -> float:
    """frac times the oracle's stability limit for the shot's largest velocity."""
    import oracle
    return frac * oracle.dt_max(spec.space_order, inputs.H, spec.vmax)


def eta_for(spec) -> np.ndarray:
    """The oracle's default damping rounded to float32 (the exact array both
    sides then consume)."""
    import oracle
    return oracle.default_damping(spec.m, spec.nbl, inputs.H).astype(np.float32)


def run_gpu(spec, nt, dt, eta=None, sources=None, chunks=None, state=None, **opts):
    """Run nt steps through the C-ABI; returns (u^n, u^{n-1}, Shot)."""
    shot = fd.Shot(spec.interior, spec.space_order, inputs.H, dt, spec.nbl, **opts)
    shot.set_model(spec.m, eta)
    for (src, wav) in (sources if sources is not None else
                       [(spec.source, inputs.ricker(spec.f0, dt, spec.nt))]):
        shot.inject(*src, wav)
    if state is not None:
        shot.load_state(*state)
    for n in (chunks or [nt]):
        shot.forward(n)
    return shot.wavefield(0), shot.wavefield(1), shot


def run_oracle(oracle, spec, nt, dt, eta, sources=None, state=None):
    """Same shot on the FP64 oracle; sources are interior nodes (offset by nbl)."""
    srcs = sources if sources is not None else [(spec.source, inputs.ricker(spec.f0, dt, spec.nt))]
    nodes = [tuple(c + spec.nbl for c in s) for s, _ in srcs]
    ld = max(len(w) for _, w in srcs) if srcs else 0
    wav = np.zeros((len(srcs), max(ld, 1)))
    for i, (_, w) in enumerate(srcs):
        wav[i, :len(w)] = np.asarray(w, dtype=np.float32).astype(np.float64)
    kw = {}
    if state is not None:
        kw = dict(u0=state[0].astype(np.float64), u_prev0=state[1].astype(np.float64), step0=state[2])
    return oracle.forward(spec.m.astype(np.float64), None if eta is None else eta.astype(np.float64),
                          spec.space_order, inputs.H, dt, nt, nodes, wav, **kw)


def rel_l2(a, b) -> float:
    b = np.asarray(b, dtype=np.float64)
    d = np.asarray(a, dtype=np.float64) - b
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(d) / nb) if nb > 0 else float(np.linalg.norm(d))
