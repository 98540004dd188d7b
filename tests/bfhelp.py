"""Helpers shared by the GPU parity tests (no arithmetic of the method here)."""
import contextlib
import importlib.util
import os

import numpy as np
import torch


def normwise(X, R, rows):
    """Max over problems of ||X - R||_F / ||R||_F on the first `rows` rows."""
    X = np.asarray(X)[:, :, :rows]
    R = np.asarray(R)[:, :, :rows]
    num = np.sqrt(np.sum((X - R) ** 2, axis=(1, 2)))
    den = np.sqrt(np.sum(R ** 2, axis=(1, 2)))
    den = np.where(den == 0, 1.0, den)
    return float(np.max(num / den)) if X.shape[0] else 0.0


def lower_part(X, n):
    """Column-major batch (b, ncols, ld) -> its lower triangle (zeros above), first n rows."""
    X = np.array(X[:, :n, :n])
    for j in range(n):
        X[:, j, :j] = 0.0
    return X


@contextlib.contextmanager
def forced(bf, routine, code, variant, p0=0, p1=0, p2=0, p3=0):
    """The variant at every batch size (no small-batch switch), for the duration of a block."""
    bf.tune_set(routine, code, 0, 1 << 30, variant | bf.TUNE_FORCE, p0, p1, p2, p3)
    try:
        yield
    finally:
        bf.reset_table()


def gpu(x):
    return torch.as_tensor(x).to("cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def build_lib():
    """Build libbfgpu.so (loading the build script by path) and import the binding."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location(
        "bfgpu_build", os.path.join(root, "paper_1902_08115_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()
    import paper_1902_08115_gb300 as bf
    return bf
