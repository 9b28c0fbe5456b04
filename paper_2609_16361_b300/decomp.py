"""z-slab decomposition of one periodic domain: the split a multi-device run of the sweep uses
(streaming moves one population per field across a z-face per step), here driven on one device.

A slab of nz_s interior planes is an ordinary periodic domain of nz_s + 2 planes: ghost plane 0
below and nz_s + 1 above, initialised with the whole domain's planes z0 - 1 .. z0 + nz_s
(periodic wrap).  Before every step the ghost planes receive the only values an interior cell
pulls from them: the +z population of the lower neighbour's top interior plane (into ghost
plane 0) and the -z population of the upper neighbour's bottom interior plane (into the top
ghost plane), for the five fields.  Interior cells then evolve exactly as in the undivided
domain.  `SlabSet` runs this with the C ABI (grlb_halo_exchange_z) for slabs on one device;
`SlabRank` is one slab per rank of a multi-device run, its slices packed into device buffers
(grlb_halo_pack_z), swapped with the neighbouring ranks by `ring_exchange` (torch.distributed
point-to-point send / receive: NCCL between devices, gloo between CPU ranks) and unpacked into
the ghost planes (grlb_halo_unpack_z); `exchange_planes` is the rule on host population arrays
(35 planes of nx ny nz, x fastest), for checks on the CPU.
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


def slab_params(prm):
    """A slab keeps two buffers: of moments when the case stores moments (streaming 2), else
    of populations."""
    return prm.replace(streaming=2 if prm.streaming == 2 else 0)


def halo_values(prm) -> int:
    """Values per cell of one exchanged slab face: the population along z of each field, or
    Q_k / 8 and J*_k,z of each field for moment storage."""
    return 10 if prm.streaming == 2 else 5


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
        self.doms = [capi.Domain(slab_params(p.params), stream=stream) for p in self.parts]

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


def ring_exchange(top, bottom, rank: int, world: int):
    """The ghost slices of this rank's slab in a periodic ring of z-slabs, one slab per rank
    (rank r owns the planes above rank r - 1's).  Sends `top` (the +z populations of the top
    interior plane) to rank r + 1 and `bottom` (the -z populations of the bottom interior plane)
    to rank r - 1, both mod world, and returns (from_below, from_above): rank r - 1's top and
    rank r + 1's bottom, the values of this slab's ghost planes 0 and nz - 1.  One rank closes
    the ring on itself (no communication).  Point-to-point operations of one batch are matched
    in the order they are issued, so with two ranks (the same peer above and below) the first
    send meets the first receive."""
    if world == 1:
        return top, bottom
    import torch
    import torch.distributed as dist
    up, down = (rank + 1) % world, (rank - 1) % world
    from_below = torch.empty_like(top)
    from_above = torch.empty_like(bottom)
    ops = [dist.P2POp(dist.isend, top, up), dist.P2POp(dist.isend, bottom, down),
           dist.P2POp(dist.irecv, from_below, down), dist.P2POp(dist.irecv, from_above, up)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    return from_below, from_above


class SlabRank:
    """This rank's z-slab of a periodic domain split over `world` ranks, one device each: the
    slab's own domain on the current device, and before every step its outgoing slices packed
    on the device, swapped with the neighbouring ranks by ring_exchange and unpacked into its
    ghost planes.  All of it runs on `stream` (a torch stream; NCCL orders its transfers after
    the packing and the unpacking after them), so the interior evolves bitwise as the
    undivided domain's planes z0 .. z0 + nzs - 1."""

    def __init__(self, case: inputs.Case | None, rank: int, world: int, stream=None, sizes=None,
                 part: inputs.Case | None = None):
        """case: the whole domain, split by `sizes` (default: even slabs); or part: this rank's
        slab (with its ghost planes, as slab_case builds it) when the whole domain is too large
        to build on one host."""
        import torch
        from . import capi
        self.capi = capi
        self.rank, self.world = rank, world
        if part is None:
            prm = case.params
            self.sizes = list(sizes) if sizes is not None else slab_sizes(prm.nz, world)
            self.z0 = slab_starts(self.sizes)[rank]
            self.part = slab_case(case, self.z0, self.sizes[rank])
        else:
            self.part = part
            self.z0 = part.meta.get("z0", 0)
        prm = self.part.params
        self.stream = stream or torch.cuda.Stream()
        self.dom = capi.Domain(slab_params(self.part.params), stream=self.stream.cuda_stream)
        nxy = prm.nx * prm.ny
        dtype = torch.float32 if prm.storage == inputs.STORE_F32 else torch.int16  # raw 16-bit values
        self.top = torch.empty((halo_values(prm), nxy), dtype=dtype, device="cuda")
        self.bottom = torch.empty_like(self.top)
        self.nx, self.ny = prm.nx, prm.ny

    def init(self, ce_init: bool | None = None):
        p = self.part
        self.dom.init(p.rho, p.u, p.p, ce_init=ce_init)

    def init_device(self, rho, u, p):
        """Initialise from the slab's fields already on the device (torch FP64 tensors)."""
        self.capi.grlb_init_primitive_device(self.dom.h, rho.data_ptr(), u.data_ptr(), p.data_ptr())

    def step(self, n: int = 1):
        import torch
        c = self.capi
        with torch.cuda.stream(self.stream):
            for _ in range(n):
                c.grlb_halo_pack_z(self.dom.h, self.top.data_ptr(), self.bottom.data_ptr())
                below, above = ring_exchange(self.top, self.bottom, self.rank, self.world)
                c.grlb_halo_unpack_z(self.dom.h, below.data_ptr(), above.data_ptr())
                self.dom.step(1)

    def conserved_interior(self) -> np.ndarray:
        return interior(self.dom.conserved(), self.nx, self.ny)

    def close(self):
        self.dom.close()


def allreduce_sum(values: np.ndarray) -> np.ndarray:
    """Sum of a small FP64 vector over the ranks of the default torch.distributed group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(np.asarray(values, dtype=np.float64))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.numpy()
