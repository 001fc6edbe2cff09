"""Helpers shared by the GPU parity tests: the CUDA library (built in-tree),
oracle structures built from the same workloads dicts, relative errors."""
import numpy as np

from oracle import retrieval as ort
from paper_1501_01752_b300 import build

K0 = 2 * np.pi


def gsm():
    build.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1501_01752_b300 import gsm as g
    return g


def oracle_structure(st):
    return ort.Structure(st["periods"], st.get("eps_host", 1.0), st.get("shapes", ()), st.get("voxels"))


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))
