"""Shared test helpers: move seeded workloads to the device and compare with the oracle."""
import numpy as np


def to_device(lsq, mat, dtype="f64", with_f64=False, ld_pad=0):
    """workloads dict -> (api.Matrix, keepalive list, the FP64 values the oracle must see)."""
    import torch
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    keep = []
    if mat["kind"] == "dense":
        A = np.asarray(mat["A"], dtype=np.float64)
        m, n = A.shape
        ld = n + ld_pad
        T = torch.zeros(m, ld, dtype=tdt, device="cuda")
        T[:, :n] = torch.from_numpy(A).to("cuda").to(tdt)
        view = T[:, :n] if ld_pad else T
        f64 = None
        if with_f64:
            f64 = torch.zeros(m, ld, dtype=torch.float64, device="cuda")
            f64[:, :n] = T[:, :n].double()
            keep.append(f64)
        keep.append(T)
        Mx = lsq.Matrix(view if not ld_pad else T[:, :n], vals_f64=f64)
        seen = T[:, :n].double().cpu().numpy()
        return Mx, keep, {"kind": "dense", "A": seen}
    rp = torch.from_numpy(np.asarray(mat["row_ptr"], np.int64)).cuda()
    ci = torch.from_numpy(np.asarray(mat["col_idx"], np.int32)).cuda()
    v = torch.from_numpy(np.asarray(mat["vals"], np.float64)).cuda().to(tdt)
    f64 = v.double() if with_f64 else None
    keep += [rp, ci, v] + ([f64] if f64 is not None else [])
    Mx = lsq.Matrix(row_ptr=rp, col_idx=ci, vals=v, n=mat["n"], vals_f64=f64)
    seen = dict(mat)
    seen["vals"] = v.double().cpu().numpy()
    return Mx, keep, seen


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)
