"""Shared set-up for the GPU parity tests (inputs from the seeded
generators; expected values from the FP64 oracle only)."""

import numpy as np

import oracle
from paper_1405_4524_gb300 import inputs


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rel_per_source(a, b):
    n = a.shape[0]
    return [rel(a[k], b[k]) for k in range(n)]


def random_spinors(dims, n, seed):
    X, Y, Z, T = dims
    rng = np.random.default_rng(seed)
    sh = (n, T, Z, Y, X, 4, 3)
    return rng.standard_normal(sh) + 1j * rng.standard_normal(sh)


def device_buffer(nbytes):
    import torch

    return torch.empty(max(int(nbytes), 16), dtype=torch.uint8, device="cuda")


class Setup:
    """A lattice with links loaded into a context and its oracle data."""

    def __init__(self, dims, eps=0.25, seed=1001, recon=12, t_bc=-1):
        from paper_1405_4524_gb300 import stochq

        self.sq = stochq
        self.dims = tuple(dims)
        self.t_bc = t_bc
        self.U = inputs.make_links(dims, eps, seed)
        self.F = oracle.field_strength(self.U)
        self.par = oracle.parity_field(dims)
        self.ctx = stochq.sq_create(dims, t_bc)
        stochq.sq_load_gauge(self.ctx, self.U, recon)

    def close(self):
        if self.ctx:
            self.sq.sq_destroy(self.ctx)
            self.ctx = None

    def Ainv(self, kappa, csw):
        return np.linalg.inv(oracle.clover_matrices(self.F, kappa, csw))
