"""Sharded resampling on the GPU (smc_shard_reduce / smc_shard_ancestors).

A population cut into W slices of whole tiles is resampled slice by slice: the
slices' tile records, concatenated in slice order, are all any slice needs of
the others.  Every slice's call must give the bits smc_resample gives for the
whole population: its ancestors on the offsets it owns, S and the log-Z
increment, and the near-boundary count summed over the slices; the owned
ranges must partition [0, N) in slice order and hold exactly the offsets whose
ancestors lie in the slice.  Emulated here as W slices on one GPU in one
process (the kernels of different slices never wait on one another), and end
to end through shard.resample with two gloo ranks sharing the GPU."""
import os
import socket

import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu

TILE = 4096


def _logw(N, case, seed):
    lw = inputs.random_logw(N, seed=seed, scale=2.0, dead_frac=0.2)
    if case == "heavy":
        lw[np.random.default_rng(seed).integers(0, N, 3)] += 15.0
    elif case == "dead_first":
        lw[: min(N, 2 * TILE)] = -np.inf
    elif case == "one":
        lw[:] = -np.inf
        lw[N // 2] = -3.0
    elif case == "dead":
        lw[:] = -np.inf
    elif case == "equal":
        lw[:] = 0.75
    if not np.isfinite(lw).any() and case != "dead":
        lw[0] = 0.0
    return lw


def _sharded(lw, u, W):
    """Every slice's records and search on one GPU; returns the assembled
    ancestors, each slice's (lo, hi), out3 and n_near."""
    import torch
    from paper_2112_00364_gb300 import shard, smc

    N = lw.shape[0]
    x = torch.from_numpy(lw).cuda()
    sl = shard.slices(N, W)
    recs = [smc.shard_reduce(x[f:f + n]) for f, n in sl]
    rec_all = torch.cat(recs)
    assert rec_all.numel() == 16 * (-(-N // TILE))
    anc = torch.full((N,), -1, dtype=torch.int32, device="cuda")
    out = []
    for f, n in sl:
        _, rng, o3, nn = smc.shard_ancestors(x[f:f + n], f, rec_all, N, u, ancestors=anc)
        torch.cuda.synchronize()
        out.append((tuple(int(v) for v in rng.cpu()), o3.cpu().numpy(), int(nn.cpu()[0])))
    return anc.cpu().numpy(), sl, out


@pytest.mark.parametrize("N,W", [(2 * TILE, 2), (3 * TILE + 1234, 2), (5 * TILE + 17, 3),
                                 (16 * TILE, 5), (100_003, 4), ((1 << 22) + 999, 8)])
@pytest.mark.parametrize("case", ["plain", "heavy", "dead_first", "one", "equal", "dead"])
def test_shard_equals_whole_resample(N, W, case):
    import torch
    from paper_2112_00364_gb300 import smc

    lw = _logw(N, case, N + W)
    u = 0.6180339887498949
    a_s, sl, per = _sharded(lw, u, W)
    a_w, o3_w, nn_w = smc.resample(torch.from_numpy(lw).cuda(), u)
    torch.cuda.synchronize()
    a_w, o3_w = a_w.cpu().numpy(), o3_w.cpu().numpy()
    np.testing.assert_array_equal(a_s, a_w)
    for _, o3, _ in per:  # the same exact integers on every slice
        np.testing.assert_array_equal(o3, o3_w)
    assert sum(nn for _, _, nn in per) == int(nn_w.cpu()[0])
    ranges = [r for r, _, _ in per]
    assert ranges[0][0] == 0 and ranges[-1][1] == N
    assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
    for (f, n), (lo, hi) in zip(sl, ranges):
        assert np.all((a_s[lo:hi] >= f) & (a_s[lo:hi] < f + n))
    if case == "dead":
        np.testing.assert_array_equal(a_s, np.arange(N))


def test_shard_matches_oracle():
    N = 3 * TILE + 77
    lw = _logw(N, "plain", 5)
    u = 0.25
    a_s, _, per = _sharded(lw, u, 3)
    a_o, flag, incr, m, S, rc = oracle.resample(lw, u)
    assert rc == 0
    diff = a_s != a_o
    assert np.all(flag[diff] == 1)
    o3 = per[0][1]
    assert abs(o3[2] - incr) <= 1e-12 * max(1.0, abs(incr))


def test_shard_argument_checks():
    import torch
    from paper_2112_00364_gb300 import smc

    N = 3 * TILE
    x = torch.zeros(N, dtype=torch.float64, device="cuda")
    rec = smc.shard_reduce(x)
    for first, n in [(100, TILE), (0, TILE - 1), (2 * TILE, 2 * TILE)]:
        with pytest.raises(smc.SmcError) as e:
            smc.shard_ancestors(x[:n] if first == 0 else x[TILE:TILE + n], first, rec, N, 0.5)
        assert e.value.status == smc.EINVAL
    with pytest.raises(smc.SmcError):
        smc.shard_reduce(x[:0])


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, N, q):
    import torch
    import torch.distributed as dist

    from paper_2112_00364_gb300 import shard, smc

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        torch.cuda.set_device(0)
        lw = _logw(N, "heavy", 3)
        x = torch.from_numpy(lw).cuda()
        state = torch.stack([torch.arange(N, dtype=torch.float64) * 3 + f for f in range(4)]).cuda()
        first, n = shard.slices(N, ws)[rank]
        new, o3, n_near, (lo, hi) = shard.resample(x[first:first + n], state[:, first:first + n],
                                                   first, N, 0.77)
        a_w, o3_w, nn_w = smc.resample(x, 0.77)
        want = state[:, a_w.long()[first:first + n]]
        torch.cuda.synchronize()
        ok = (torch.equal(new, want) and torch.equal(o3.cpu(), o3_w.cpu())
              and n_near == int(nn_w.cpu()[0]))
        q.put((rank, bool(ok), lo, hi))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_shard_resample_two_ranks_one_gpu():
    import torch.multiprocessing as mp

    N = 5 * TILE + 321
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, N, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=300) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    assert all(ok for _, ok, _, _ in got)
    assert got[0][2] == 0 and got[0][3] == got[1][2] and got[1][3] == N
