"""Reference jet post-processing (test infrastructure): connected components
of the liquid phi > threshold with face connectivity, merged across periodic
faces, and the breakup length / drop statistics derived from them (Sec. 6:
breakup length L_b, drop size d_e).  Written with scipy.ndimage.label and a
union-find over the periodic face pairs; shares no code with the CUDA path.
"""
from __future__ import annotations

import numpy as np


def components(phi, threshold, periodic):
    """phi: array [n_last, ..., n_x] with the jet axis first (3D: [nz][ny][nx],
    2D: [ny][nx]); periodic: per array axis, whether it wraps.  Returns a list
    of (cells, lo, hi) with lo / hi the extent along axis 0."""
    from scipy import ndimage
    liquid = phi > threshold
    lab, n = ndimage.label(liquid, structure=ndimage.generate_binary_structure(liquid.ndim, 1))
    parent = list(range(n + 1))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for ax, wrap in enumerate(periodic):
        if not wrap:
            continue
        first = np.take(lab, 0, axis=ax)
        last = np.take(lab, lab.shape[ax] - 1, axis=ax)
        for a, b in zip(first.ravel(), last.ravel()):
            if a and b:
                ra, rb = find(int(a)), find(int(b))
                if ra != rb:
                    parent[max(ra, rb)] = min(ra, rb)
    roots = np.array([find(k) for k in range(n + 1)])
    merged = roots[lab]
    out = []
    for r in sorted(set(roots[1:].tolist())):
        idx = np.nonzero(merged == r)[0] if merged.ndim == 1 else np.nonzero(merged == r)
        along = idx[0]
        out.append((int(along.size), int(along.min()), int(along.max())))
    return out


def jet_stats(phi, threshold, periodic, dim):
    comps = components(phi, threshold, periodic)
    jet = None
    for k, (v, lo, hi) in enumerate(comps):
        if lo == 0 and (jet is None or v > comps[jet][0]):
            jet = k
    drops = [v for k, (v, lo, hi) in enumerate(comps) if k != jet]
    diam = [2.0 * np.sqrt(v / np.pi) if dim == 2 else np.cbrt(6.0 * v / np.pi) for v in drops]
    return dict(n_components=len(comps), has_jet=int(jet is not None),
                breakup_length=float(comps[jet][2] + 1) if jet is not None else 0.0,
                n_drops=len(drops), mean_drop_diameter=float(np.mean(diam)) if drops else 0.0,
                drop_volume=float(sum(drops)), drop_volumes=sorted(drops))
