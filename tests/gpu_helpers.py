"""Helpers shared by the GPU tests: run the CUDA path through the C ABI on a
synthetic workload and measure its error against the FP64 oracle."""
import numpy as np

import oracle
from paper_2301_09662_gb300 import epic


def torch_inputs(wl, device="cuda"):
    import torch
    v = torch.from_numpy(np.ascontiguousarray(wl.v)).to(device)
    g = None if wl.gains is None else torch.from_numpy(np.ascontiguousarray(wl.gains)).to(device)
    return v, g


def run_gpu(wl, precision=epic.EPIC_FP32, flags=0, T=None, plan=None):
    import torch
    p = plan or epic.Plan.from_workload(wl, precision=precision, flags=flags)
    v, g = torch_inputs(wl)
    if T is not None:
        v = v[:T].contiguous()
    out = p.image(v, g)
    torch.cuda.synchronize()
    assert p.status() == epic.EPIC_OK
    return out.cpu().numpy().astype(np.complex128), p


def peak_rel_err(gpu, ref, grid_n, P):
    """Per channel: max |I_gpu - I_ref| over pixels and products, divided by the
    channel's peak max(|XX|, |YY|) of the reference (the error metric)."""
    errs = []
    for a, b in zip(oracle.split_channels(gpu, grid_n, P), oracle.split_channels(ref, grid_n, P)):
        peak = np.max(np.abs(b[:2])) if P == 2 else np.max(np.abs(b[0]))
        errs.append(np.max(np.abs(a - b)) / peak)
    return np.array(errs)
