"""A battery of small runs through every kernel family of the library, for the bounds-checked
build (libgrlb_checked.so): each scenario's accesses must all fall inside live regions, and each
scenario's results are digested so that the same battery on the plain library can be compared
with them bit for bit.

    GRLB_LIB=<library> python tests/checked_battery.py <out.json>

Writes <out.json> = {"checked": bool, "scenarios": {name: {"parts": {label: {"digest": sha,
"narrays": n}}, "violations": n, "first": addr}}, "probe": [...], "final": counts} and
<out.npz> with each part's floating-point arrays under "scenario|label|i".  Run as a child process (the library a process loads is fixed
at its first call) by tests/test_gpu_checked.py.
"""
import dataclasses
import hashlib
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2609_16361_b300 import capi, decomp, inputs, mms, serve  # noqa: E402

STORAGES = (inputs.STORE_F32, inputs.STORE_F16, inputs.STORE_BF16)
COLLISIONS = (inputs.COLL_BGK, inputs.COLL_RLB_SENSOR, inputs.COLL_RLB_GATED)


def with_params(case, **kw):
    return dataclasses.replace(case, params=case.params.replace(**kw))


class Digest:
    """Per part of a scenario (one part per run): the sha256 of its arrays and the floating-point
    arrays themselves (FP64 copies, for sizing a difference when two digests differ)."""

    def __init__(self):
        self.parts = {}
        self.cur = None

    def part(self, label):
        self.cur = self.parts.setdefault(label, {"h": hashlib.sha256(), "arrays": []})

    def add(self, *arrays):
        if self.cur is None:
            self.part("all")
        for a in arrays:
            a = np.ascontiguousarray(a)
            assert a.dtype.kind in "biuf", a.dtype  # numbers only: an object array digests addresses
            self.cur["h"].update(a.tobytes())
            if a.dtype.kind == "f":
                self.cur["arrays"].append(a.astype(np.float64).ravel())

    def add_diag(self, g):
        self.add(np.array([g[k] for k in ("totals",)]).ravel(),
                 np.array([g["ke"], g["eps_s"], g["eps_d"], g["rho_min"], g["p_min"],
                           g["n_floor"], g["n_nan"], g["n_sensor"], g["step"]], dtype=np.float64))

    def result(self):
        return {k: {"digest": v["h"].hexdigest(), "narrays": len(v["arrays"])}
                for k, v in self.parts.items()}

    def arrays(self, scenario):
        return {f"{scenario}|{k}|{i}": a for k, v in self.parts.items() for i, a in enumerate(v["arrays"])}


def run_domain(dg, case, steps, ce=None, stream=None):
    prm = case.params
    dg.part(f"{prm.name} {prm.nx}x{prm.ny}x{prm.nz} s{prm.storage} c{prm.collision} "
            f"aa{prm.streaming} n{steps} ce{int(bool(ce))}")
    d = capi.Domain(case.params, stream=stream)
    d.init(case.rho, case.u, case.p, ce_init=ce)
    d.step(steps)
    d.step_diag()
    dg.add_diag(d.diag(allow_nonfinite=True))
    dg.add(d.conserved())
    rho, u, p, T = d.primitive()
    dg.add(rho, u, p, T)
    d.close()


def sc_sweeps(dg):
    """Every storage x collision on a tiled grid (32^3: 32 x 4 CTA tiles) and on the linear
    mapping (40 x 21 x 7, ragged last brick); 9 sweeps (one graph replay of 8) + 1 diagnostic.
    And rows of whole bricks (128 x 4 x 6), where the plain library's 16-bit sweeps prefetch the
    bricks two planes ahead into L2 and the checked build does not: the results must not move."""
    for s in STORAGES:
        for c in COLLISIONS:
            run_domain(dg, with_params(inputs.tgv3d(32, storage=s), collision=c), 9)
            run_domain(dg, inputs.random_smooth(40, 21, 7, seed=3, storage=s, collision=c), 9)
        run_domain(dg, inputs.random_smooth(128, 4, 6, seed=7, storage=s), 9)


def sc_one_buffer(dg):
    """One-buffer (AA) streaming: periodic boxes and an X_DIRICHLET_EQ tube (outflow record),
    after odd and even step counts (the readback gathers after odd ones)."""
    for s in (inputs.STORE_F32, inputs.STORE_F16):
        for steps in (4, 5):
            for case in (inputs.tgv3d(16, storage=s), inputs.sod(64, storage=s)):
                run_domain(dg, with_params(case, streaming=1), steps)


def sc_tubes(dg):
    """Dirichlet-ghost tubes, two buffers: Sod, Becker, the double rarefaction (floors)."""
    run_domain(dg, inputs.sod(80), 12)
    run_domain(dg, inputs.becker(128, ny=4, nz=4), 12)
    run_domain(dg, inputs.double_rarefaction(64), 12)


def sc_ce_init(dg):
    run_domain(dg, inputs.tgv3d(16, mach=0.5, re=100.0), 3, ce=True)
    run_domain(dg, inputs.sod(64), 3, ce=True)
    run_domain(dg, with_params(inputs.tgv3d(16, storage=inputs.STORE_F16), streaming=1), 3, ce=True)


def sc_source(dg):
    import torch
    c = mms.case(8)
    d = capi.Domain(c.params)
    d.init(c.rho, c.u, c.p)
    S = torch.zeros((5, c.params.ncells), dtype=torch.float32, device="cuda")
    capi.grlb_set_source_device(d.h, S.data_ptr())
    for k in range(3):
        S.copy_(torch.from_numpy(mms.source(8, (k + 0.5) * c.params.dt)).float())
        torch.cuda.synchronize()
        d.step(1)
    capi.grlb_set_source_device(d.h, None)
    d.step(1)
    capi.grlb_set_source_device(d.h, S.data_ptr())  # still set when the domain goes
    d.step(1)
    dg.add(d.conserved())
    d.close()


def sc_staging_and_checkpoint(dg):
    a, b = inputs.tgv3d(16), inputs.tgv3d(16, mach=0.8)
    d = capi.Domain(a.params)
    capi.grlb_stage_primitive(d.h, a.rho, a.u, a.p)
    capi.grlb_stage_primitive(d.h, b.rho, b.u, b.p)
    capi.grlb_init_from_stage(d.h)
    d.step(3)
    blob = capi.grlb_save(d.h)
    capi.grlb_init_from_stage(d.h)
    capi.grlb_load(d.h, blob)
    d.step(2)
    dg.add(d.conserved())
    capi.grlb_stage_primitive(d.h, a.rho, a.u, a.p)  # staged, never consumed
    d.close()


def sc_init_device(dg):
    import torch
    c = inputs.random_smooth(24, 8, 6, seed=4)
    d = capi.Domain(c.params)
    t = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (c.rho, c.u, c.p)]
    capi.grlb_init_primitive_device(d.h, *(x.data_ptr() for x in t))
    torch.cuda.synchronize()
    d.step(2)
    dg.add(d.conserved())
    d.close()


def batch_cases():
    out = []
    for i, s in enumerate((inputs.STORE_F32, inputs.STORE_F16)):
        out.append(inputs.sod(96 + 40 * i, storage=s))
        out.append(inputs.becker(160 + 32 * i, ny=4, nz=4, storage=s))
        out.append(inputs.tgv3d(16 + 4 * i, storage=s, re=100.0))
        out.append(inputs.random_smooth(37, 5, 3, seed=i, storage=s, collision=COLLISIONS[i]))
    return out


def sc_batches(dg):
    for sched in (capi.SCHED_CONCURRENT, capi.SCHED_TABLE_CONST, capi.SCHED_TABLE):
        for tile in (0, 1, 32, 128):
            if sched == capi.SCHED_CONCURRENT and tile:
                continue
            dg.part(f"schedule {sched} tile {tile}")
            cases = batch_cases()
            doms = [capi.Domain(c.params) for c in cases]
            for d, c in zip(doms, cases):
                d.init(c.rho, c.u, c.p)
            b = capi.grlb_batch_create([d.h for d in doms], schedule=sched, max_lanes=2)
            if tile:
                capi.grlb_batch_set_tile_x(b, [tile] * len(doms))
            capi.grlb_batch_step(b, 5)
            active = [1 if i % 3 else 0 for i in range(len(doms))]
            capi.grlb_batch_set_active(b, active)
            capi.grlb_batch_step(b, 3)
            capi.grlb_batch_destroy(b)
            for d in doms:
                dg.add(d.conserved())
                d.close()


def sc_serve(dg):
    trace = inputs.serving_trace(seed=5, n_requests=6, rate=500.0, tgv_range=(12, 16), steps_range=(10, 40))
    dg.part("served")
    for r in serve.Server(chunk=8, keep_fields=True).run(trace, realtime=False):
        dg.add(np.frombuffer(r.digest.encode(), dtype=np.uint8), r.fields)


def sc_slabs(dg):
    c = inputs.random_smooth(24, 6, 16, seed=2)
    s = decomp.SlabSet(c, [7, 9])
    s.init()
    s.step(4)
    dg.add(s.conserved())
    s.close()
    r = decomp.SlabRank(inputs.tgv3d(16, storage=inputs.STORE_F16), 0, 1)
    r.init()
    r.step(3)
    dg.add(r.conserved_interior())
    r.close()
    mc = with_params(inputs.tgv3d(16), streaming=2)   # moment slabs: Q_k, J*_k,z exchanged
    s = decomp.SlabSet(mc, [7, 9])
    s.init()
    s.step(3)
    dg.add(s.conserved())
    s.close()
    r = decomp.SlabRank(mc, 0, 1)
    r.init()
    r.step(3)
    dg.add(r.conserved_interior())
    r.close()


def sc_check_finite(dg):
    import torch
    c = inputs.tgv3d(16)
    d = capi.Domain(c.params)
    d.init(c.rho, c.u, c.p)
    dev = torch.zeros(1, dtype=torch.int32, device="cuda")
    host = torch.zeros(1, dtype=torch.int32).pin_memory()
    capi.grlb_check_finite(d.h, dev.data_ptr())
    capi.grlb_check_finite(d.h, host.data_ptr())
    torch.cuda.synchronize()
    dg.add(dev.cpu().numpy(), host.numpy())
    d.close()


def sc_noalloc(dg):
    import torch
    for s in (inputs.STORE_F32, inputs.STORE_BF16):
        c = inputs.random_smooth(40, 21, 7, seed=9, storage=s)
        d = capi.Domain(c.params)
        d.init(c.rho, c.u, c.p)
        d.step(2)
        state = capi.grlb_save(d.h)[32:]
        fa = torch.from_numpy(state.copy()).cuda()
        fb = torch.zeros_like(fa)
        diag = torch.zeros(13, dtype=torch.float64, device="cuda")
        capi.grlb_step_diag_noalloc(c.params, fa.data_ptr(), fb.data_ptr(), diag.data_ptr(), None)
        torch.cuda.synchronize()
        dg.add(fb.cpu().numpy(), diag.cpu().numpy())
        d.close()


def spectral_sums(sums):
    """The three sums of a spectral call as numbers (a dict itself would digest as an object)."""
    return np.array([sums["eps_s"], sums["eps_d"], sums["ke_u"]])


def sc_spectral(dg):
    cases = [inputs.tgv3d(16), with_params(inputs.tgv3d(32, storage=inputs.STORE_F16), streaming=1),
             inputs.tgv2d(32), inputs.tgv2d(64), inputs.tgv2d(512)]
    for i, c in enumerate(cases):
        dg.part(f"spectral {c.params.nx}x{c.params.ny}x{c.params.nz} s{c.params.storage} aa{c.params.streaming}")
        d = capi.Domain(c.params)
        d.init(c.rho, c.u, c.p)
        d.step(3 if c.params.streaming else 1 + i % 2)  # odd: the one-buffer readback gathers
        E, sums = d.spectral()
        dg.add(np.asarray(E), spectral_sums(sums))
        d.close()


def sc_read_cells(dg):
    """Point probes in the three layouts (two buffers; one buffer after even and after odd
    steps, with the outflow record of a tube)."""
    for case in (inputs.random_smooth(40, 21, 7, seed=3), inputs.sod(64)):
        for streaming, steps in ((0, 3), (1, 2), (1, 3)):
            dg.part(f"cells {case.params.name} aa{streaming} n{steps}")
            d = capi.Domain(case.params.replace(streaming=streaming))
            d.init(case.rho, case.u, case.p)
            d.step(steps)
            dg.add(capi.grlb_read_cells(d.h, np.arange(case.params.ncells)))
            d.close()


def sc_moments(dg):
    """Moment storage: the sweep (tiled and linear launches, Dirichlet ghosts), its diagnostic
    sweep, the Chapman-Enskog start, readback, probes and spectra."""
    for case, ce in ((inputs.tgv3d(16), False), (inputs.tgv3d(16, mach=0.5, re=100.0), True),
                     (inputs.tgv3d(32), False),   # tiled: the column-marching sweep
                     (inputs.random_smooth(128, 8, 6, seed=8), False),   # whole-brick rows: L2 prefetch
                     (inputs.random_smooth(40, 21, 7, seed=3), False), (inputs.sod(64), False)):
        run_domain(dg, with_params(case, streaming=2), 9, ce=ce)
        d = capi.Domain(case.params.replace(streaming=2))
        d.init(case.rho, case.u, case.p)
        d.step(2)
        dg.add(capi.grlb_read_cells(d.h, np.arange(case.params.ncells)))
        if case.params.name.startswith("tgv"):
            E, sums = d.spectral()
            dg.add(np.asarray(E), spectral_sums(sums))
        d.close()


def sc_ffma(dg):
    import torch
    sink = torch.zeros(4 * 256, dtype=torch.float32, device="cuda")
    capi.grlb_ffma_probe(4, 2, sink.data_ptr())
    torch.cuda.synchronize()
    dg.add(sink.cpu().numpy())


SCENARIOS = [sc_sweeps, sc_one_buffer, sc_tubes, sc_ce_init, sc_source, sc_staging_and_checkpoint,
             sc_init_device, sc_batches, sc_serve, sc_slabs, sc_check_finite, sc_noalloc, sc_spectral,
             sc_read_cells, sc_moments, sc_ffma]


def probe_checker():
    """The checker's own test: ranges inside, at the edges of, straddling and outside a region
    made live for the probe (addresses compared, never accessed)."""
    import torch
    t = torch.empty(256, dtype=torch.float32, device="cuda")
    base = t.data_ptr()
    cases = [(0, 4, 0), (1020, 4, 0), (0, 1024, 0), (1024, 4, 1), (-4, 4, 1), (1022, 4, 1), (512, 1024, 1)]
    out = []
    for off, nbytes, expect in cases:
        before = capi.grlb_check_read()["violations"]
        capi.grlb_check_probe(base, 1024, off, nbytes)
        got = capi.grlb_check_read()["violations"] - before
        out.append({"offset": off, "bytes": nbytes, "expected": expect, "counted": got})
    capi.grlb_check_read(reset=True)
    return out


def main(path):
    import torch
    torch.cuda.init()
    checked = capi.grlb_checked_build()
    result = {"checked": checked, "library": capi.LIB_PATH, "scenarios": {}}
    arrays = {}
    if checked:
        result["probe"] = probe_checker()
    for sc in SCENARIOS:
        dg = Digest()
        v0 = capi.grlb_check_read()["violations"] if checked else 0
        sc(dg)
        torch.cuda.synchronize()
        entry = {"parts": dg.result()}
        arrays.update(dg.arrays(sc.__name__))
        if checked:
            cnt = capi.grlb_check_read()
            entry["violations"] = cnt["violations"] - v0
            entry["first"] = cnt["first_addr"]
        result["scenarios"][sc.__name__] = entry
    if checked:
        result["final"] = capi.grlb_check_read()
    np.savez(os.path.splitext(path)[0] + ".npz", **arrays)
    with open(path, "w") as f:
        json.dump(result, f, indent=1)


if __name__ == "__main__":
    main(sys.argv[1])
