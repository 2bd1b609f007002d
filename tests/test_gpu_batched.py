"""Batched Cholesky-type refinement (lyap_solve_ir_batched): equations of uneven order
and rank solved concurrently, each to the normalised residual of Eq. (4.1) <= 1e-12,
matching the oracle's exact solution and the lone lyap_solve_ir results, with one failing
equation reported without stopping the others."""
import numpy as np
import pytest

import lyapgen as gen
import oracle as O
from tests.gpu_util import N, T

pytestmark = pytest.mark.gpu


def lib():
    from paper_2510_02126_gb300 import lyap
    return lyap


def test_batched_matches_single_and_oracle():
    lp = lib()
    eqs = gen.batch_uneven(count=12, nmin=24, nmax=160, rmax=6, seed=gen.SEED_BASE + 50)
    o = lp.make_opts(u_s="fp16", tau_ir=1e-12, imax=20)
    Zs, infos, st = lp.solve_ir_batched([T(e["A"]) for e in eqs], [T(e["L"]) for e in eqs], opts=o, workers=4)
    assert st == 0
    for k, (e, Z, inf) in enumerate(zip(eqs, Zs, infos)):
        assert inf.converged, k
        res = lp.residual(T(e["A"]), T(e["L"]), Z)
        assert res <= 1e-12, (k, res)
        Z1, _, inf1 = lp.solve_ir(T(e["A"]), T(e["L"]), opts=o)
        X, X1 = N(Z) @ N(Z).T, N(Z1) @ N(Z1).T
        assert np.linalg.norm(X - X1) <= 1e-10 * np.linalg.norm(X1), k
        if k < 3:
            Xo = O.bartels_stewart(e["A"], e["L"] @ e["L"].T)
            assert np.linalg.norm(X - Xo) <= 1e-10 * np.linalg.norm(Xo), k


def test_batched_reports_a_failing_equation():
    lp = lib()
    eqs = gen.batch_uneven(count=5, nmin=24, nmax=64, rmax=3, seed=gen.SEED_BASE + 51)
    As = [e["A"] for e in eqs]
    As[2] = -As[2]  # not Hurwitz: the sign iteration does not reach -I
    o = lp.make_opts(u_s="fp16", tau_ir=1e-12, imax=10)
    Zs, infos, st = lp.solve_ir_batched([T(a) for a in As], [T(e["L"]) for e in eqs], opts=o, workers=3,
                                        raise_on_error=False)
    assert st < 0
    assert infos[2].status < 0
    for k in (0, 1, 3, 4):
        assert infos[k].status >= 0 and infos[k].converged, k


def test_batched_on_fresh_contexts_after_destroyed_ones():
    # Worker contexts created after earlier contexts were destroyed receive recycled device
    # memory: every status word must be cleared before its first read (regression: a stale
    # nonzero word aborted solves with a random status or cut the first Newton solve short).
    import gc

    lp = lib()
    # the batched workload family (32 equations, n 64..1017, rank 1..8), all of which
    # converge in at most 7 FP16-inner refinement steps
    eqs = gen.batch_uneven(count=32, nmin=64, nmax=1024, rmax=8)
    As, Ls = [T(e["A"]) for e in eqs], [T(e["L"]) for e in eqs]
    o = lp.make_opts(u_s="fp16", tau_ir=1e-12, imax=10)
    try:
        for rep in range(3):
            if lp._ctx is not None:
                lp._ctx.close()
                lp._ctx = None
            gc.collect()
            Zs, infos, st = lp.solve_ir_batched(As, Ls, opts=o, workers=8, raise_on_error=False)
            assert st == 0, (rep, st)
            for k, inf in enumerate(infos):
                assert inf.converged and inf.res_final <= 1e-12, (rep, k, inf.status, inf.res_final)
    finally:
        if lp._ctx is not None:
            lp._ctx.close()
            lp._ctx = None


def test_batched_full_config_256():
    # the batched workload at full size: 256 equations, n log-uniform in [64, 1024], rank 1..8,
    # FP16 inner solves, FP64 refinement to 1e-12 (imax = 10, as the bench).  Every equation
    # converges (residual of Eq. (4.1) from the factors); a seeded sample of 16 equals the lone
    # lyap_solve_ir result and the oracle's Bartels-Stewart solution
    lp = lib()
    eqs = gen.batch_uneven(count=256, nmin=64, nmax=1024, rmax=8)
    o = lp.make_opts(u_s="fp16", tau_ir=1e-12, imax=10)
    Zs, infos, st = lp.solve_ir_batched([T(e["A"]) for e in eqs], [T(e["L"]) for e in eqs], opts=o, workers=8)
    assert st == 0
    assert all(inf.converged for inf in infos)
    assert max(inf.res_final for inf in infos) <= 1e-12
    for k in gen.rng(gen.SEED_BASE + 52).choice(256, size=16, replace=False):
        e, Z = eqs[k], Zs[k]
        X = N(Z) @ N(Z).T
        Z1, _, inf1 = lp.solve_ir(T(e["A"]), T(e["L"]), opts=o)
        X1 = N(Z1) @ N(Z1).T
        assert np.linalg.norm(X - X1) <= 1e-10 * np.linalg.norm(X1), k
        Xo = O.bartels_stewart(e["A"], e["L"] @ e["L"].T)
        assert np.linalg.norm(X - Xo) <= 1e-10 * np.linalg.norm(Xo), k
