"""Row-sharded sampling on the GPU: the device phases (lsq_shard_colmax, _colsum, _weights,
_draw) run for each row block of a matrix in turn, as the ranks of the multi-GPU design
would, with the collectives done here on the host (MAX of the column maxima, SUM of the
limbs, the offsets from the gathered totals, MAX merge of the draws).  The merged indices and
probabilities and every rank's column scales must equal lsq_sample_rows on the whole matrix
bit for bit."""
import numpy as np
import pytest
import torch

import workloads as W
from helpers import to_device

pytestmark = pytest.mark.gpu


def _blocks(mat, world):
    m = mat["A"].shape[0] if mat["kind"] == "dense" else mat["m"]
    b = [m * r // world for r in range(world + 1)]
    out = []
    for r in range(world):
        r0, r1 = b[r], b[r + 1]
        if mat["kind"] == "dense":
            out.append((r0, {"kind": "dense", "A": np.ascontiguousarray(mat["A"][r0:r1])}))
        else:
            rp = mat["row_ptr"]
            out.append((r0, {"kind": "csr", "m": r1 - r0, "n": mat["n"], "row_ptr": rp[r0:r1 + 1] - rp[r0],
                             "col_idx": mat["col_idx"][rp[r0]:rp[r1]], "vals": mat["vals"][rp[r0]:rp[r1]]}))
    return out


@pytest.mark.parametrize("case,world,sampling,normalize", [
    ("dense", 2, 0, 1), ("csr", 3, 0, 1), ("udv", 4, 0, 1), ("csr", 2, 1, 1), ("dense", 3, 0, 0)])
def test_sharded_sampling_equals_one_process(lsq, case, world, sampling, normalize):
    mat = {"dense": lambda: W.gaussian_dense(6001, 70, 3),
           "csr": lambda: W.sparse_random(30000, 400, 8, 5),
           "udv": lambda: W.udv_dense(20000, 96, 1e4, 2)}[case]()
    if case == "dense":
        mat["A"] *= np.logspace(-3, 3, mat["A"].shape[0])[:, None]   # rows of very different norms
    o = lsq.opts(seed=41, sampling=sampling, normalize=normalize)
    Mx, keep, seen = to_device(lsq, mat)
    idx_ref, p_ref, d_ref = lsq.lsq_sample_rows(Mx, o)
    s = idx_ref.numel()
    ranks = []
    for r0, blk in _blocks(mat, world):
        Ml, kl, _ = to_device(lsq, blk)
        ranks.append((r0, Ml, kl))
    colmax = torch.stack([lsq.shard_colmax(Ml) for _, Ml, _ in ranks]).amax(dim=0)
    limbs = torch.stack([lsq.shard_colsum(Ml, colmax) for _, Ml, _ in ranks]).sum(dim=0)
    parts = [lsq.shard_weights(Ml, colmax, limbs, o) for _, Ml, _ in ranks]
    for d, _, _ in parts:
        assert torch.equal(d, d_ref)
    W_all = np.stack([Wr for _, _, Wr in parts])
    idx = torch.full((s,), -1, dtype=torch.int32, device="cuda")
    p = torch.zeros(s, dtype=torch.float64, device="cuda")
    owned = 0
    for r, ((r0, Ml, _), (_, prefix, _)) in enumerate(zip(ranks, parts)):
        off, tot = lsq.shard_offsets(W_all, r)
        ir, pr = lsq.shard_draw(prefix, r0, off, tot, s, o)
        owned += int((ir >= 0).sum())
        idx = torch.maximum(idx, ir)
        p = p + pr
    torch.cuda.synchronize()
    assert owned == s
    assert torch.equal(idx, idx_ref)
    assert torch.equal(p, p_ref)
