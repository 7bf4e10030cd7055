"""Helpers shared by the GPU parity tests (host-side marshalling only)."""
import numpy as np
import torch


def rel_err(got, ref):
    ref = np.asarray(ref)
    scale = np.abs(ref).max()
    return float(np.abs(np.asarray(got) - ref).max() / (scale if scale > 0 else 1.0))


def to_dev(s, arr, dtype=torch.float64, level=0):
    """numpy (ns, n) -> device [ns][stride] of the solver's layout."""
    arr = np.atleast_2d(arr)
    t = s.stage_vector(ns=arr.shape[0], dtype=dtype, level=level)
    t[:, :arr.shape[1]] = torch.from_numpy(np.ascontiguousarray(arr)).to(dtype)
    return t


def from_dev(t, n):
    torch.cuda.synchronize()
    return t[:, :n].double().cpu().numpy()
