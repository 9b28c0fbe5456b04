"""z-slab decomposition of one periodic domain: the split a multi-device run of the sweep uses
(streaming moves one population per field across a z-face per step), here driven on one device.

A slab of nz_s interior planes is an ordinary periodic domain of nz_s + 2 planes: ghost plane 0
below and nz_s + 1 above, initialised with the whole domain's planes z0 - 1 .. z0 + nz_s
(periodic wrap).  Before every step the ghost planes receive the only values an interior cell
pulls from them: the +z population of the lower neighbour's top interior plane (into ghost
plane 0) and the -z population of the upper neighbour's bottom interior plane (into the top
ghost plane), for the five fields.  Interior cells then evolve exactly as in the undivided
domain.  `SlabSet` runs this with the C ABI (grlb_halo_exchange_z); `exchange_planes` is the
same rule on host population arrays (35 planes of nx ny nz, x fastest), for checks on the CPU
and for ranks that exchange slices over torch.distributed.
"""
from __future__ import annotations

import numpy as np

from . import inputs

PZ, MZ = 5, 6  # links +z and -z


def slab_sizes(nz: int, nslabs: int) -> list[int]:
    """Interior planes per slab, as even as possible (each >= 1)."""
    if not 1 <= nslabs <= nz:
        raise ValueError("need 1 <= nslabs <= nz")
    base, extra = divmod(nz, nslabs)
    return [base + (1 if i < extra else 0) for i in range(nslabs)]


def slab_starts(sizes) -> list[int]:
    return [int(v) for v in np.concatenate([[0], np.cumsum(sizes)[:-1]])]


def slab_case(case: inputs.Case, z0: int, nzs: int) -> inputs.Case:
    """The slab of interior planes z0 .. z0 + nzs - 1 with one ghost plane on each side."""
    prm = case.params
    if prm.bc != inputs.BC_PERIODIC:
        raise ValueError("z-slabs split periodic domains")
    nx, ny, nz = prm.nx, prm.ny, prm.nz
    planes = np.arange(z0 - 1, z0 + nzs + 1) % nz

    def take(a):
        return np.ascontiguousarray(a.reshape(nz, ny * nx)[planes].reshape(-1))

    u = np.stack([take(case.u[k]) for k in range(3)])
    sp = prm.replace(nz=nzs + 2, name=f"{prm.name}-z{z0}+{nzs}")
    return inputs.Case(sp, take(case.rho), u, take(case.p), dict(case.meta, z0=z0, nzs=nzs))


def interior(Q: np.ndarray, nx: int, ny: int) -> np.ndarray:
    """Interior planes of a slab field array (..., (nzs + 2) nx ny) -> (..., nzs nx ny)."""
    nxy = nx * ny
    return Q[..., nxy:Q.shape[-1] - nxy]


def stitch(parts) -> np.ndarray:
    """Whole-domain arrays (..., N) from slab interiors in z order."""
    return np.concatenate(list(parts), axis=-1)


def top_slice(f: np.ndarray, nxy: int) -> np.ndarray:
    """+z populations of the top interior plane (5, nxy) of a slab's populations (35, M)."""
    nzl = f.shape[1] // nxy
    return np.stack([f[7 * k + PZ, (nzl - 2) * nxy:(nzl - 1) * nxy] for k in range(5)])


def bottom_slice(f: np.ndarray, nxy: int) -> np.ndarray:
    """-z populations of the bottom interior plane (5, nxy)."""
    return np.stack([f[7 * k + MZ, nxy:2 * nxy] for k in range(5)])


def put_bottom_ghost(f: np.ndarray, nxy: int, s: np.ndarray):
    for k in range(5):
        f[7 * k + PZ, 0:nxy] = s[k]


def put_top_ghost(f: np.ndarray, nxy: int, s: np.ndarray):
    nzl = f.shape[1] // nxy
    for k in range(5):
        f[7 * k + MZ, (nzl - 1) * nxy:nzl * nxy] = s[k]


def exchange_planes(f_lower: np.ndarray, f_upper: np.ndarray, nxy: int):
    """The ghost exchange between two adjacent slabs' host populations, in place."""
    put_bottom_ghost(f_upper, nxy, top_slice(f_lower, nxy))
    put_top_ghost(f_lower, nxy, bottom_slice(f_upper, nxy))


class SlabSet:
    """A periodic domain as z-slabs on the current CUDA device, stepped with the ghost exchange
    of the C ABI before every step (two-buffer streaming)."""

    def __init__(self, case: inputs.Case, sizes, stream=None):
        from . import capi
        self.capi = capi
        self.case = case
        self.sizes = list(sizes)
        if len(self.sizes) < 2 or sum(self.sizes) != case.params.nz:
            raise ValueError("slab sizes must add up to nz, at least two slabs")
        self.parts = [slab_case(case, z0, n) for z0, n in zip(slab_starts(self.sizes), self.sizes)]
        self.doms = [capi.Domain(p.params.replace(streaming=0), stream=stream) for p in self.parts]

    def init(self, ce_init: bool | None = None):
        for d, p in zip(self.doms, self.parts):
            d.init(p.rho, p.u, p.p, ce_init=ce_init)

    def step(self, n: int = 1):
        S = len(self.doms)
        for _ in range(n):
            for i in range(S):
                self.capi.grlb_halo_exchange_z(self.doms[i].h, self.doms[(i + 1) % S].h)
            for d in self.doms:
                d.step(1)

    def conserved(self) -> np.ndarray:
        prm = self.case.params
        return stitch(interior(d.conserved(), prm.nx, prm.ny) for d in self.doms)

    def interior_totals(self) -> list[np.ndarray]:
        prm = self.case.params
        return [interior(d.conserved(), prm.nx, prm.ny).sum(axis=1) for d in self.doms]

    def close(self):
        for d in self.doms:
            d.close()
        self.doms = []


def allreduce_sum(values: np.ndarray) -> np.ndarray:
    """Sum of a small FP64 vector over the ranks of the default torch.distributed group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(np.asarray(values, dtype=np.float64))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.numpy()
