"""The exchange step of a population sharded over ranks (host logic, CPU, gloo).

A population of N particles sharded in whole tiles over W ranks is resampled by
all-gathering the tiles' records, searching on every rank the offsets whose
ancestors lie in its own slice, and sending the states of those ancestors to
the ranks whose slices hold the new indices (Section 3.3's resampling step,
split at its one global dependency).  Here the ancestors come from the oracle's
systematic resampling of the whole population; the test checks that the slices
are whole tiles, that the records arrive in rank order, and that after the
exchange every rank holds exactly state[:, ancestors[its slice]] of the whole
population, for W = 2 and 3, FP64 and int32 fields, ragged last slices and
ancestor ranges that cross one or several slices."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

TILE = 4096


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _population(N: int, case: str, seed: int):
    rng = np.random.default_rng(seed)
    logw = rng.normal(0.0, 1.0, N)
    if case == "heavy":  # a few particles own most of the mass: long runs of equal ancestors
        logw[rng.integers(0, N, 5)] += 12.0
    elif case == "dead_slice":  # the first slice has no weight at all: its offsets all move
        logw[: 2 * TILE] = -np.inf
    elif case == "one":  # one survivor (in the ragged last slice): every offset copies it
        logw[:] = -np.inf
        logw[N - 1] = 0.0
    else:
        logw[rng.integers(0, N, 20)] = -np.inf
    return logw


def _rank(rank: int, ws: int, port: int, N: int, case: str, q):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2112_00364_gb300 import shard

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        sl = shard.slices(N, ws)
        first, n = sl[rank]
        logw = _population(N, case, 11)
        anc, _, _, _, _, rc = oracle.resample(logw, 0.3141)
        assert rc == 0
        # records: stand-ins of this rank's tiles (16 bytes each, rank-tagged)
        nt = -(-n // TILE)
        rec = torch.arange(16 * nt, dtype=torch.int64).remainder(251).to(torch.uint8) + rank
        got = shard.gather_records(rec)
        want = torch.cat([torch.arange(16 * (-(-nq // TILE)), dtype=torch.int64)
                          .remainder(251).to(torch.uint8) + r for r, (_, nq) in enumerate(sl)])
        assert torch.equal(got, want)
        # the offsets this rank's tiles own: ancestors in [first, first + n)
        lo = int(np.searchsorted(anc, first, side="left"))
        hi = int(np.searchsorted(anc, first + n, side="left"))
        ar = np.arange(N)
        for dtype in (torch.float64, torch.int32):
            state = torch.stack([torch.tensor(ar * 7 + f, dtype=torch.int64) for f in range(3)]).to(dtype)
            local = state[:, first:first + n]
            produced = local[:, torch.from_numpy(anc[lo:hi].astype(np.int64) - first)]
            new = shard.exchange_states(produced, lo, hi, sl)
            expect = state[:, torch.from_numpy(anc[first:first + n].astype(np.int64))]
            assert new.dtype == dtype and new.shape == (3, n)
            assert torch.equal(new, expect)
        moved = (hi - lo) - max(0, min(hi, first + n) - max(lo, first))
        q.put((rank, first, n, lo, hi, moved))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def _run(ws: int, N: int, case: str):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, N, case, q)) for r in range(ws)]
    for p in procs:
        p.start()
    got = []
    try:
        got = sorted(q.get(timeout=180) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    return got


@pytest.mark.parametrize("ws,N,case", [
    (2, 3 * TILE + 1234, "plain"),
    (2, 4 * TILE, "heavy"),
    (3, 5 * TILE + 17, "dead_slice"),
    (3, 3 * TILE + 1, "one"),
])
def test_exchange_gloo(ws, N, case):
    got = _run(ws, N, case)
    # the searched ranges partition [0, N) in rank order
    assert got[0][3] == 0 and got[-1][4] == N
    assert all(a[4] == b[3] for a, b in zip(got, got[1:]))
    if case == "dead_slice":  # rank 0 owns no weight: all its new particles come from others
        assert got[0][3] == got[0][4] and got[1][5] > 0
    if case == "one":  # the survivor's rank searched every offset
        assert [r[4] - r[3] for r in got] == [0, 0, N]


def test_slices_whole_tiles():
    from paper_2112_00364_gb300 import shard

    for N in (1, TILE, TILE + 1, 7 * TILE - 5, 100_000, 1 << 20):
        for ws in (1, 2, 3, 4, 8):
            sl = shard.slices(N, ws)
            assert len(sl) == ws and sum(n for _, n in sl) == N
            pos = 0
            for r, (first, n) in enumerate(sl):
                if n:
                    assert first == pos and first % TILE == 0
                    if first + n < N:
                        assert n % TILE == 0
                pos += n
            tiles = [-(-n // TILE) for _, n in sl]
            assert max(tiles) - min(tiles) <= 1
