"""One step of a sampled node from the patch around it.

One lattice Boltzmann step moves information at most two nodes: a node's
post-step populations are pulled from its neighbours' post-collision ones,
and a collision reads phi (a sum over the node's own g) at the neighbours.
So the oracle, run for one step on the (2R+1)-node patch (cube in 3D) around
a node, reproduces that node's step exactly when R >= 2 and the patch's own
faces cannot reach it:
  * interior nodes: a periodic patch (its wrapped edges are R nodes away);
  * nodes within R of the low (high) face of the last axis: a patch flush
    with that face, carrying the face's real condition, with a wall (or, on
    the inlet side, the outflow the inlet needs) on its far side, more than
    R nodes from the node.
The other axes are periodic in the workloads this serves, so their patch
indices wrap exactly.  Used by the full-size parity tests (GPU state) and
pinned on the CPU against the oracle's own full-grid step.
"""
import numpy as np

import lbm_cases as C

R = 3


def patch_params(p, z, y, x, kind):
    """(oracle parameters of the patch, index vectors (zz, yy, xx) into the
    grid, position (cz, cy, cx) of the node in the patch)."""
    q = dict(p)
    bc = list(p["bc"])
    D3 = p["lattice"] == C.D3Q19
    nz, ny, nx = p.get("nz", 1), p["ny"], p["nx"]
    w = 2 * R + 1
    xx = (x - R + np.arange(w)) % nx
    if D3:
        yy = (y - R + np.arange(w)) % ny
        n, a, ilo, ihi = nz, z, 4, 5
    else:
        yy = None
        n, a, ilo, ihi = ny, y, 2, 3
    if kind == "interior":
        mm, cm = (a - R + np.arange(w)) % n, R
        lo = hi = C.PERIODIC
    elif kind == "low":
        mm, cm = np.arange(w), a
        lo = bc[ilo]
        hi = C.OUTFLOW if lo == C.INLET else C.WALL
    else:
        mm, cm = n - w + np.arange(w), a - (n - w)
        lo, hi = C.WALL, bc[ihi]
    if D3:
        q.update(nx=w, ny=w, nz=w, bc=[C.PERIODIC] * 4 + [lo, hi])
        if p.get("inlet_radius", 0.0) > 0.0:
            q["inlet_center"] = [p["inlet_center"][0] - (x - R), p["inlet_center"][1] - (y - R)]
        return q, (mm, yy, xx), (cm, R, R)
    q.update(nx=w, ny=w, nz=1, bc=[C.PERIODIC, C.PERIODIC, lo, hi, C.PERIODIC, C.PERIODIC])
    return q, (np.zeros(1, np.int64), mm, xx), (0, cm, R)


def node_step(orc, p, z, y, x, kind, get_patch):
    """The oracle's post-step (f, g) at node (z, y, x): get_patch(idx)
    returns the pre-step (f, g) float64 arrays [Q][len zz][len yy][len xx]
    over the index vectors idx."""
    q, idx, (cz, cy, cx) = patch_params(p, z, y, x, kind)
    o = orc.Oracle(q)
    try:
        f, g = get_patch(idx)
        o.set_populations(f, g)
        o.step(1)
        rf, rg = o.populations()
    finally:
        o.close()
    return rf[:, cz, cy, cx], rg[:, cz, cy, cx]


def samples_jet(p, r, n_interior=40):
    nz, ny, nx = p["nz"], p["ny"], p["nx"]
    cx, cy = p["inlet_center"]
    s = [(int(r.integers(R, nz - R)), int(r.integers(ny)), int(r.integers(nx)), "interior")
         for _ in range(n_interior)]
    # the inlet plane and the two above it, inside, across and outside the nozzle
    rn = p["inlet_radius"]
    for k, f in enumerate((-1.5, -1.05, -0.55, 0.0, 0.55, 1.0, 1.25, -1.25, 0.2, -0.2, 0.75, -0.75)):
        s.append((k % 3, int(round(cy + f * rn)) % ny, int(round(cx - 0.5 * f * rn)) % nx, "low"))
    for k in range(9):
        s.append((nz - 1 - (k % 3), int(r.integers(ny)), int(r.integers(nx)), "high"))
    return s


def samples_walls2d(p, r, n_interior=40):
    ny, nx = p["ny"], p["nx"]
    s = [(0, int(r.integers(R, ny - R)), int(r.integers(nx)), "interior") for _ in range(n_interior)]
    s += [(0, k % 3, int(r.integers(nx)), "low") for k in range(9)]
    s += [(0, ny - 1 - (k % 3), int(r.integers(nx)), "high") for k in range(9)]
    return s
