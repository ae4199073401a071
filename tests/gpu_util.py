"""Helpers shared by the GPU tests: device problems from NumPy inputs."""
import numpy as np

from paper_2502_03749_gb300 import pins


def torch_cuda():
    import torch
    return torch


def dev(x, dtype=None):
    torch = torch_cuda()
    t = torch.as_tensor(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda().contiguous()


def dense_device_problem(C, a, b):
    torch = torch_cuda()
    Ct = dev(C, torch.float32 if C.dtype == np.float32 else torch.float64)
    return pins.make_problem("dense", dev(a), dev(b), C=Ct, on_device=True)


def random_state(m, n, seed, eta=0.05, s=2.0, kind="dense32"):
    """Costs in [0,1] (float32-representable when kind == 'dense32'), positive
    marginals, and potentials after a few oracle Sinkhorn steps (realistic z)."""
    from oracle import pins_oracle as po
    rng = np.random.default_rng(seed)
    C = rng.uniform(0, 1, size=(m, n))
    if kind == "dense32":
        C = C.astype(np.float32).astype(np.float64)
    a = rng.uniform(0.5, 1.5, size=m); a /= a.sum()
    b = rng.uniform(0.5, 1.5, size=n); b /= b.sum()
    F, G = np.zeros(m), np.zeros(n)
    for _ in range(3):
        F, _ = po.sinkhorn_row_step(C, a, F, G, eta, s)
        G = po.sinkhorn_col_step(C, b, F, G, eta, s)
    F = F + rng.normal(size=m) * 0.01 * eta
    G = G + rng.normal(size=n) * 0.01 * eta
    return C, a, b, F, G, eta, s
