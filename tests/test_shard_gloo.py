"""Row-sharded sampling with world-size-2 and -3 gloo ranks on CPU (the host steps of the
multi-GPU design; no GPU).  Each rank holds a contiguous block of rows; its weight prefix
comes from the oracle on its own rows (row weights are row-local once the column scales are
known).  The library's host code then does the rest: the offsets from the all-gathered
totals and the filtered draws; the ranks merge by MAX.  The merged indices must equal the
oracle's single-process draws on the whole matrix, bit for bit."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _limbs(v):
    return np.array([(v >> (32 * k)) & 0xFFFFFFFF for k in range(4)], np.int64)


def _rank(rank, world, port, case, out_dir):
    import datetime
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import oracle
    import workloads as W
    from paper_1806_02968_gb300 import _lib
    _lib.load()
    from paper_1806_02968_gb300 import api
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    mat = W.gaussian_dense(3001, 40, 7) if case == "dense" else W.sparse_random(5000, 300, 8, 3)
    full = oracle.Sample(mat, seed=17)
    m = full.mat.m
    bounds = [m * r // world for r in range(world + 1)]
    r0, r1 = bounds[rank], bounds[rank + 1]
    if mat["kind"] == "dense":
        local = {"kind": "dense", "A": np.ascontiguousarray(mat["A"][r0:r1])}
    else:
        rp = mat["row_ptr"]
        local = {"kind": "csr", "m": r1 - r0, "n": mat["n"], "row_ptr": rp[r0:r1 + 1] - rp[r0],
                 "col_idx": mat["col_idx"][rp[r0]:rp[r1]], "vals": mat["vals"][rp[r0]:rp[r1]]}
    w_lo, w_hi = oracle.row_weights(local, full.inv_d2)
    P_lo, P_hi = oracle.prefix(w_lo, w_hi)
    prefix = np.stack([P_lo, P_hi], axis=1).reshape(-1)
    Wr = (int(P_hi[-1]) << 64) | int(P_lo[-1])
    # all-gather of the ranks' totals (four 32-bit limbs each)
    got = [torch.zeros(4, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(got, torch.from_numpy(_limbs(Wr)))
    W_all = torch.stack(got).numpy()
    off, tot = api.shard_offsets(W_all, rank)
    idx = api.shard_draw_host(prefix, r0, off, tot, seed=17, t0=0, s=full.s)
    t = torch.from_numpy(idx.astype(np.int64))
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    dist.destroy_process_group()
    np.save(os.path.join(out_dir, f"merged{rank}.npy"), t.numpy())
    np.save(os.path.join(out_dir, "single.npy"), full.idx)
    own = int((idx >= 0).sum())
    with open(os.path.join(out_dir, f"own{rank}.txt"), "w") as f:
        f.write(f"{own}\n")


@pytest.mark.parametrize("world,case", [(2, "dense"), (3, "csr")])
def test_sharded_draws_equal_one_process(tmp_path, world, case):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, case, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    single = np.load(tmp_path / "single.npy")
    owns = [int(open(tmp_path / f"own{r}.txt").read()) for r in range(world)]
    assert sum(owns) == single.size and all(o > 0 for o in owns)   # each draw has one owner
    for r in range(world):
        merged = np.load(tmp_path / f"merged{r}.npy")
        assert np.array_equal(merged, single.astype(np.int64))


def test_offsets_carry_across_limbs(lsq):
    """Totals near 2^64 and 2^96: the offsets and the grand total keep every carry."""
    vals = [(1 << 64) - 5, (1 << 96) + 123456789, 7, (1 << 127) // 3]
    W_all = np.stack([_limbs(v) for v in vals])
    for r in range(len(vals)):
        off, tot = lsq.shard_offsets(W_all, r)
        back = lambda l: sum(int(l[k]) << (32 * k) for k in range(4))
        assert back(off) == sum(vals[:r]) and back(tot) == sum(vals)
