"""Helpers shared by the GPU tests: build/load the library once, move numpy
inputs to the device, relative L-infinity error."""

import numpy as np


def ensure_built():
    from paper_2404_14864_gb300 import build, kfbi
    build.build()
    return kfbi.lib()


def dev(a):
    import torch
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a).to("cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel_linf(a, ref):
    ref = np.asarray(ref)
    return float(np.abs(np.asarray(a) - ref).max() / max(np.abs(ref).max(), 1e-300))
