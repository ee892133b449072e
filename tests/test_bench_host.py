"""Host-side logic of bench.py: the replicas' max-over-ranks timing (gloo, 2 ranks on CPU)
and the algorithmic byte model."""
import os
import socket

import pytest

import bench
import synth as S


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank  # the slower rank decides
    m = bench.max_over_ranks(ms)
    q.put((rank, m, bench.replica_value(2048, 100, world, m)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for _, m, v in res:
        assert m == 15.0
        assert v == pytest.approx(2 * 2048 * 2048 * 100 / 0.015)


def test_max_over_ranks_without_group():
    assert bench.max_over_ranks(3.5) == 3.5


def test_algorithmic_byte_model_production():
    m = bench.algorithmic_bytes(S.island2048_dleith(), True)
    n, K = 2048, 682
    I = n * (K + 1) * 8
    assert m["row_stage"] == (3, 14 * I)
    step = sum(a * b for a, b in m.values())
    assert 1.2e9 < step < 1.3e9


def test_full_field_model_counts_per_closure():
    """Full-field round-trip model: 2 U_N per 2-D transform plus stage I/O; per step, with island and sponge:
    none 60, Smagorinsky 84, Leith 72, dynamic Smagorinsky 147, dynamic Leith 123 U_N."""
    import dataclasses
    base = S.island2048_dleith()
    un = base.n * base.n * 4
    expect = {S.NONE: (5, 60), S.SMAG: (9, 84), S.LEITH: (7, 72), S.DSMAG: (18, 147), S.DLEITH: (14, 123)}
    for kind, (row, step) in expect.items():
        wl = dataclasses.replace(base, closure=kind)
        assert bench.field_model_bytes(wl, True) == (row * un, step * un)
    # each stage: the transforms' round trips (2 U_N each) plus 4 (static) or 7 (dynamic) U_N of stage I/O
    ninv = {S.NONE: 4, S.SMAG: 6, S.LEITH: 4, S.DSMAG: 12, S.DLEITH: 8}
    nfwd = {S.NONE: 1, S.SMAG: 3, S.LEITH: 3, S.DSMAG: 6, S.DLEITH: 6}
    for kind, per_stage in bench.FIELD_TRAVERSALS_PER_STAGE.items():
        io = 7 if kind in (S.DSMAG, S.DLEITH) else 4
        assert per_stage == 2 * (ninv[kind] + nfwd[kind]) + io
    row, step = bench.field_model_bytes(base, True)
    assert abs(step - 2.064e9) < 1e6 and abs(row - 234.9e6) < 1e5


def test_ab2cn_byte_model_at_2048_dynamic_leith():
    """One explicit evaluation per step: 38 mixed arrays, 13 spectra and the two factor fields (Eq. 4)."""
    wl = S.island2048_dleith()
    n, K = wl.n, (wl.n - 1) // 3
    I, Sp, R = n * (K + 1) * 8, (K + 1) * (2 * K + 1) * 8, n * n * 4
    model = bench.algorithmic_bytes_ab2cn(wl, True)
    assert sum(a * b for a, b in model.values()) == 38 * I + 13 * Sp + 2 * R
    assert all(a == 1 for a, _ in model.values())


def test_series_pair_count_matches_the_oracle_nan_pattern():
    import numpy as np
    import oracle as O
    les = np.zeros((5, 2))
    ff = np.zeros((7, 2))
    dist, _ = O.lag_table(les, ff, -3, 4)
    assert bench.valid_pairs(5, 7, -3, 4) == int(np.sum(~np.isnan(dist)))


def test_ensemble_shards_partition_the_members():
    for world in (1, 2, 3, 4, 8):
        shards = [bench.ensemble_shard(96, r, world) for r in range(world)]
        flat = sorted(i for sh in shards for i in sh)
        assert flat == list(range(96))
        sizes = [len(sh) for sh in shards]
        assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("kind", [S.NONE, S.SMAG, S.LEITH, S.DSMAG, S.DLEITH])
def test_torch_fft_context_step_is_the_oracle_step(kind):
    """The torch.fft form timed beside libqg computes the oracle's step (run here on the CPU in FP64)."""
    import numpy as np
    import torch
    import oracle as O
    wl = S.Workload("t", 48, "island", beta=5.0, U=0.5, closure=kind, c=0.2, radius=0.8, seed=1)
    ts = bench.TorchFFTStep(wl, dtype=torch.float64, device="cpu")
    w0 = S.init_field(1, 48, k_peak=16)
    wh = ts.project(torch.from_numpy(w0))
    ref = O.QGOracle(48, wl.L, wl.beta, wl.U, wl.mask(), wl.sponge_field(), O.Closure(kind, c=0.2), O.Params())
    ref.set_state(w0)
    for _ in range(5):
        wh = ts.step(wh)
    ref.step(5)
    a, b = ts.inv(wh).numpy(), ref.get_state()
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-12


def test_transform_counts_per_step():
    """Real 2-D transforms per step, (x passes + y passes) / 2 over the launch sequence: the RK3 table's dynamic
    Leith entry (3 stages x (8 inverse + 6 forward) + Brinkman 4 + sponge 2) and the AB2CN count (one evaluation)."""
    import bench
    import synth as S
    wl = S.island2048_dleith()
    assert bench.transforms_per_step(wl, 0) == 3 * (8 + 6) + 4 + 2
    assert bench.transforms_per_step(wl, 1) == (8 + 6) + 3 + 2
    bare = S.Workload("b", 256, "none", beta=5.0, U=0.0, closure=S.NONE, sponge=False)
    assert bench.transforms_per_step(bare, 1) == 4 + 1
    assert bench.step_flop_model(wl, 1) < bench.step_flop_model(wl, 0)
