"""Helpers shared by the GPU tests: run the same seeded problem through the
CUDA library (via its C ABI binding) and through the oracle."""
import numpy as np
import torch


def to_dev(U):
    return torch.as_tensor(np.ascontiguousarray(U), dtype=torch.float64, device="cuda")


def rel_err(gpu, ref):
    """Per variable: max |gpu - ref| / max |ref|; returns the largest.  A
    variable whose reference is only round-off (e.g. the momentum of a
    velocity component that stays zero) is measured against 1e-3 of the
    largest variable's scale instead of its own noise."""
    g = gpu.detach().cpu().numpy() if isinstance(gpu, torch.Tensor) else np.asarray(gpu)
    r = np.asarray(ref)
    floor = 1e-3 * max(float(np.abs(r[v]).max()) for v in range(r.shape[0]))
    worst = 0.0
    for v in range(r.shape[0]):
        scale = max(float(np.abs(r[v]).max()), floor)
        if scale == 0.0:
            scale = 1.0
        worst = max(worst, float(np.abs(g[v] - r[v]).max() / scale))
    return worst
