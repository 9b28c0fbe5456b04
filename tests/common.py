"""Shared helpers of the test suite (comparison norms, oracle runs, storage decode)."""
import numpy as np

WI = np.array([0.25] + [0.125] * 6)
BRICK = 128  # cells per brick of the population layout
CI = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]])


def field_scales(Q):
    """Per-field denominators: max|rho|, max|m| over all three components, max|E|."""
    mmax = np.abs(Q[1:4]).max()
    return np.array([np.abs(Q[0]).max(), mmax, mmax, mmax, np.abs(Q[4]).max()])


def rel_linf(Q, R):
    """max |Q - R| / scale per conserved field (R = reference)."""
    return np.abs(Q - R).max(axis=1) / field_scales(R)


def rel_l1(Q, R):
    """sum |Q - R| / sum |R| per field; momentum fields share the momentum-norm denominator."""
    den = np.abs(R).sum(axis=1)
    den[1:4] = np.abs(R[1:4]).sum()
    return np.abs(Q - R).sum(axis=1) / den


def run_oracle(case, steps, keep_cells=False, ce_init=False):
    import oracle
    o = oracle.Oracle(case.params)
    o.init_primitive(case.rho, case.u, case.p, ce_init=ce_init)
    o.step(steps, keep_cells=keep_cells)
    return o


def decode_populations(raw, prm, nplanes=35, cells=None):
    """FP64 populations (lattice units) from a grlb_save checkpoint, all cells or `cells`,
    as 35 rows q = 7k + i of one value per cell.

    The documented storage format: a 32-byte header, then the populations in cell bricks --
    bricks of 128 consecutive cells (storage order), each holding its 35 rows of 128 values,
    ceil(N / 128) bricks -- of deviations d = f - w_i (Q_ref + c_i . J_ref / cs^2) with
    Q_ref = (rho_ref, 0, 0, 0, p_ref/(g-1)), J_ref of m_j = p_ref e_j (lattice units), scaled by
    a per-field factor for FP16."""
    N = prm.nx * prm.ny * prm.nz
    s = prm.dt / prm.dx
    dtype = {0: np.float32, 1: np.float16, 2: np.uint16}[prm.storage]
    raw = np.frombuffer(raw, np.uint8) if isinstance(raw, bytes) else raw
    nb = (N + BRICK - 1) // BRICK
    bricks = raw[32:32 + nb * nplanes * BRICK * np.dtype(dtype).itemsize].view(dtype).reshape(nb, nplanes, BRICK)
    if cells is not None:
        cells = np.asarray(cells)
        body = bricks[cells // BRICK, :, cells % BRICK].T
    else:
        body = bricks.transpose(1, 0, 2).reshape(nplanes, nb * BRICK)[:, :N]
    if prm.storage == 2:
        d = (body.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    else:
        d = body.astype(np.float64)
    p_ref = prm.ref_p * s * s
    E_ref = p_ref / (prm.gamma - 1)
    if prm.storage == 1:
        c_ref = np.sqrt(prm.gamma * p_ref / prm.ref_rho)
        M = [prm.ref_rho, prm.ref_rho * c_ref, prm.ref_rho * c_ref, prm.ref_rho * c_ref, E_ref]
        dec = [2.0 ** -(8 - int(round(np.log2(m)))) for m in M]
    else:
        dec = [1.0] * 5
    Qref = [prm.ref_rho, 0, 0, 0, E_ref]
    f = np.empty_like(d)
    for k in range(5):
        Jref = np.zeros(3)
        if 1 <= k <= 3:
            Jref[k - 1] = p_ref
        for i in range(7):
            shift = WI[i] * (Qref[k] + 4.0 * CI[i] @ Jref)
            f[7 * k + i] = d[7 * k + i] * dec[k] + shift
    return f


def oracle_update_cells(prm, pre_of, cells):
    """The oracle's post-collision populations (35, n) of `cells` from the pre-step state:
    population i of cell x is pulled from f*_i of x - c_i (periodic wrap), or, past the ends of
    an X_DIRICHLET_EQ tube, taken from the equilibrium of the ghost state.  pre_of(cells) returns
    the pre-step populations (35, len(cells)) of any cells, e.g. the library's point probes.
    Also returns the oracle's sensor value chi per cell."""
    import oracle
    P = oracle.lattice_params(prm)
    nx, ny, nz = prm.nx, prm.ny, prm.nz
    cells = np.asarray(cells, np.int64)
    x, y, z = cells % nx, (cells // nx) % ny, cells // (nx * ny)
    src = [((x - CI[i][0]) % nx + nx * ((y - CI[i][1]) % ny + ny * ((z - CI[i][2]) % nz))) for i in range(7)]
    planes = [pre_of(src[i]) for i in range(7)]
    if prm.bc == 1:
        gl = oracle.equilibrium_state(P, list(P.left))
        gr = oracle.equilibrium_state(P, list(P.right))
        for k in range(5):
            planes[1][7 * k + 1, x == 0] = gl[7 * k + 1]       # +x population entering at x = 0
            planes[2][7 * k + 2, x == nx - 1] = gr[7 * k + 2]  # -x population entering at nx - 1
    out = np.zeros((35, cells.size))
    chi = np.zeros(cells.size)
    for n in range(cells.size):
        fhat = np.array([planes[i][7 * k + i, n] for k in range(5) for i in range(7)])
        out[:, n], info = oracle.cell(P, fhat)
        chi[n] = info.chi
    return out, chi
