"""GPU ensembles (qg_ensemble_*): members stepped together in one graph equal the same members stepped alone.

Bitwise equality with single-handle stepping (the same kernels in the same order), FP64 members against the
oracle (1e-11 relative L2), graph replay against eager launches, state changes between steps, and failure
reporting per member.  Members mix power-of-two grids (register-resident kernels) with 2^a 3^b grids (generic
kernels), both precisions, both time schemes and all closures.
"""
import math

import numpy as np
import pytest

import oracle as O
import synth as S

pytestmark = pytest.mark.gpu

qg = pytest.importorskip("paper_2508_06678_gb300")
L = 2 * math.pi


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_06678_gb300._lib import LIB_PATH
    import os
    if not os.path.exists(LIB_PATH):
        from paper_2508_06678_gb300.build import build
        build()
    qg.load()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def spec(n, kind, precision, geometry="island", scheme=0, beta=5.0, U=0.5, c=0.0):
    dt = 2e-3
    mask = S.island_mask(n, L, radius=0.8) if geometry == "island" else S.cape_mask(n, L)
    eta = 1.025 * dt if scheme == 1 else 1e-3
    return dict(n=n, precision=precision, beta=beta, U=U, mask=mask, sponge=S.sponge_mask(n, L), kind=kind, c=c,
                dt=dt, eta=eta, scheme=scheme)


MIXED = [
    spec(48, S.SMAG, qg.QG_FP64, c=0.17),
    spec(64, S.DLEITH, qg.QG_FP64, "cape", scheme=1, beta=10.0, U=1.0),
    spec(54, S.LEITH, qg.QG_FP32, c=0.25),
    spec(96, S.DSMAG, qg.QG_FP32, "cape"),
    spec(256, S.DLEITH, qg.QG_FP32),
    spec(128, S.NONE, qg.QG_FP64),
    spec(256, S.DSMAG, qg.QG_FP32, scheme=1),
]


def init(sp, seed):
    return S.init_field(seed, sp["n"], L, k_peak=max(4.0, sp["n"] / 8))


def run_alone(specs, nsteps, seeds):
    out = []
    for sp, sd in zip(specs, seeds):
        args = {k: v for k, v in sp.items() if k != "n"}
        s = qg.QGSolver(sp["n"], **args)
        s.set_state(init(sp, sd))
        s.step(nsteps)
        out.append(s.get_state())
        s.close()
    return out


def run_ensemble(specs, nsteps, seeds, chunks=(1,)):
    with qg.QGEnsemble(specs) as ens:
        for m, sp, sd in zip(ens.members, specs, seeds):
            m.set_state(init(sp, sd))
        done = 0
        for c in chunks:
            ens.step(c)
            done += c
        ens.step(nsteps - done)
        ens.sync()
        return [m.get_state() for m in ens.members]


def test_members_equal_members_stepped_alone():
    seeds = list(range(1, len(MIXED) + 1))
    a = run_ensemble(MIXED, 12, seeds)
    b = run_alone(MIXED, 12, seeds)
    for i, (x, y) in enumerate(zip(a, b)):
        assert np.array_equal(x, y), f"member {i}"


def test_fp64_members_match_the_oracle():
    specs = [spec(48, S.SMAG, qg.QG_FP64, c=0.17), spec(64, S.DLEITH, qg.QG_FP64, "cape", scheme=1),
             spec(54, S.DSMAG, qg.QG_FP64, "cape")]
    seeds = [3, 4, 5]
    got = run_ensemble(specs, 20, seeds, chunks=(1, 4))
    for sp, sd, g in zip(specs, seeds, got):
        ref = O.QGOracle(sp["n"], L, sp["beta"], sp["U"], sp["mask"], sp["sponge"], O.Closure(sp["kind"], c=sp["c"]),
                         O.Params(dt=sp["dt"], eta=sp["eta"], scheme=sp["scheme"]))
        ref.set_state(init(sp, sd))
        ref.step(20)
        assert rel(g, ref.get_state()) < 1e-11


def test_graph_replay_equals_eager(monkeypatch):
    seeds = [7] * len(MIXED)
    a = run_ensemble(MIXED, 8, seeds)
    monkeypatch.setenv("QG_NO_GRAPH", "1")
    b = run_ensemble(MIXED, 8, seeds)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_state_changes_between_steps_are_ordered():
    specs = MIXED[:5]
    with qg.QGEnsemble(specs) as ens:
        for i, (m, sp) in enumerate(zip(ens.members, specs)):
            m.set_state(init(sp, i))
        ens.step(4)
        w_new = init(specs[1], 99)
        ens.members[1].set_state(w_new)  # also restarts that member's AB2 history
        ens.step(5)
        ens.sync()
        got = [m.get_state() for m in ens.members]
    ref = run_alone([specs[1]], 5, [99])[0]
    assert np.array_equal(got[1], ref)
    ref0 = run_alone([specs[0]], 9, [0])[0]
    assert np.array_equal(got[0], ref0)


def test_nonfinite_member_is_reported_and_others_go_on():
    specs = MIXED[:4]
    with qg.QGEnsemble(specs) as ens:
        for i, (m, sp) in enumerate(zip(ens.members, specs)):
            w = init(sp, i)
            if i == 2:
                w = w.copy()
                w[3, 3] = np.nan
            m.set_state(w)
        ens.step(3)
        with pytest.raises(qg.QGError) as e:
            ens.sync()
        assert e.value.member == 2
        assert e.value.code == qg.QG_ERR_NONFINITE
        for i in (0, 1, 3):
            d = ens.members[i].diagnostics()
            assert d["finite"] and d["step"] == 3


def test_creation_error_names_the_member():
    bad = [spec(48, S.SMAG, qg.QG_FP64, c=0.17), dict(spec(48, S.SMAG, qg.QG_FP64, c=0.17), n=50,
                                                      mask=None, sponge=None)]
    with pytest.raises(qg.QGError) as e:
        qg.QGEnsemble(bad)
    assert "member 1" in str(e.value)


def test_ensemble_of_the_bench_mix_runs_and_matches_alone_for_sampled_members():
    wls = S.ensemble96()
    assert len(wls) == 96 and sorted({w.n for w in wls}) == [256, 384, 512, 768]
    pick = [0, 1, 2, 3, 50, 95]
    with qg.QGEnsemble.from_workloads(wls, precision=qg.QG_FP32) as ens:
        for m, w in zip(ens.members, wls):
            m.set_state(w.omega0())
        ens.step(3)
        ens.sync()
        got = {i: ens.members[i].get_state() for i in pick}
    for i in pick:
        w = wls[i]
        s = qg.QGSolver.from_workload(w, precision=qg.QG_FP32)
        s.set_state(w.omega0())
        s.step(3)
        assert np.array_equal(got[i], s.get_state()), i
        s.close()


@pytest.mark.parametrize("lanes,pdl,lean", [(1, 0, 0), (3, 1, 0), (2, 0, 1), (7, 1, 2)])
def test_fixed_launch_forms_equal_members_stepped_alone(lanes, pdl, lean, monkeypatch):
    """Every launch form the tuner can pick (lanes of chained members, programmatic dependent launch, the lean
    or register Germano reduction) leaves each member's arithmetic unchanged."""
    monkeypatch.setenv("QG_ENSEMBLE_LANES", str(lanes))
    monkeypatch.setenv("QG_ENSEMBLE_PDL", str(pdl))
    monkeypatch.setenv("QG_ENSEMBLE_LEAN", str(lean))
    seeds = list(range(11, 11 + len(MIXED)))
    a = run_ensemble(MIXED, 9, seeds, chunks=(1, 3))
    b = run_alone(MIXED, 9, seeds)
    for i, (x, y) in enumerate(zip(a, b)):
        assert np.array_equal(x, y), f"member {i}"


def test_tuner_choice_is_reported_cached_and_restores_the_initial_state():
    """The tuner times its candidates by stepping the members from their zero initial states, then puts them
    back: an ensemble stepped without set_state equals fresh handles stepped from zero.  A second ensemble of
    the same signature takes the choice from the cache."""
    specs = MIXED[:4]
    with qg.QGEnsemble(specs) as ens:
        cfg = ens.config()
        assert 1 <= cfg["lanes"] <= len(specs) and cfg["pdl"] in (0, 1) and cfg["lean"] in (0, 1, 2)
        assert cfg["source"] in ("timed", "cached")
        for m in ens.members:
            assert m.diagnostics()["step"] == 0
        ens.step(3)
        ens.sync()
        got = [m.get_state() for m in ens.members]
    for sp, g in zip(specs, got):
        args = {k: v for k, v in sp.items() if k != "n"}
        with qg.QGSolver(sp["n"], **args) as s:
            s.step(3)
            assert np.array_equal(g, s.get_state())
    with qg.QGEnsemble(specs) as ens2:
        assert ens2.config()["source"] == "cached"
        assert ens2.config()["lanes"] == cfg["lanes"]
