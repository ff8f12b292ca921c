"""Helpers for the GPU tests: device columns and a shared context."""
import numpy as np


def to_device(cols):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(c)).to("cuda") for c in cols]


def proof_bytes(p):
    import torch
    if isinstance(p, torch.Tensor):
        return p.cpu().numpy().tobytes()
    return np.asarray(p).tobytes()
