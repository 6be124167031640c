"""Parity rules between the CUDA path and the CPU oracle (test-side helper).

Face values: |a - b| <= REL * max(|b|, S) where S is the magnitude of the terms summed to
form the face value: the larger of the terms of the characteristic back-projection
sum_s r_s (f+_s + f-_s) (reported by the oracle) and the terms of the K-point central
flux sum_q |c_q| |F(U_q)| of the face's stencil (central_terms; where every field's
candidates are smooth the face value is that central flux, whichever way it is summed).
A face value that is small because those terms cancel is measured against the terms, as
for any floating-point sum.  How many faces need S rather than |b| is counted and logged
(strict_faces).
Flags (delta_k bits and the adaptive C_T code): identical, except where the oracle's
decision is ill-conditioned in FP64 -- its chi_k (or the adaptive beta) lies within
CUT_TOL relative of the threshold, or within NOISE_K times the sequence's rounding-noise
ratio (a characteristic sequence that is constant up to rounding, e.g. the acoustic
fields across a contact, has indicators made of rounding noise).  Faces with such a
mismatch ("switch faces") are counted and excluded from the value check.
"""
import json
import os

import numpy as np

REL = 1e-13
CUT_TOL = 1e-10
NOISE_K = 1e4


def _log(label, stats):
    """Append one JSON line of parity statistics to $TENOM_PARITY_LOG (when set)."""
    path = os.environ.get("TENOM_PARITY_LOG")
    if path:
        with open(path, "a") as fh:
            fh.write(json.dumps(dict(stats, label=label)) + "\n")


def compare_faces(Fg, flg, Fo, flo, cut, noise, scale=None, rel=REL, label="", floor=False):
    """Fg/Fo/scale: [nv, *faces]; flg/flo/cut/noise: [*faces, nv, 2].  Returns a stats dict;
    raises AssertionError on a violation.

    Value rule: |a - b| <= rel * max(|b|, S) with S the oracle's back-projection term size
    (with no S given: max(|b|, 1e-3 max|b|)).  Counts reported (and logged): switch faces,
    split into near_cutoff_faces (excused by the cutoff distance) and noise_faces (only by
    the rounding-noise ratio); strict_faces, the faces (switch faces aside) that miss
    |a - b| <= rel |b| and pass only because the value is small against its terms S (a
    face value that cancels in the back-projection sum); floor_faces, those that would
    also need the 1e-3 max|b| floor (0 is required when S is given, unless floor=True:
    for fields symmetric enough that face values vanish exactly, where both sides return
    rounding noise of terms that cancel before the back-projection)."""
    nv = Fo.shape[0]
    mism = flg != flo
    by_cut = cut <= CUT_TOL
    allowed = by_cut | (cut <= NOISE_K * noise)
    bad = mism & ~allowed
    n_bad = int(bad.sum())
    if n_bad:
        idx = np.argwhere(bad)[:5]
        info = [(tuple(i), int(flg[tuple(i)]), int(flo[tuple(i)]), float(cut[tuple(i)]), float(noise[tuple(i)]))
                for i in idx]
        raise AssertionError("%s: %d flag mismatches away from the cutoff, e.g. %s" % (label, n_bad, info))
    # faces whose flags legitimately differ are excluded from the value check
    switch = mism.reshape(mism.shape[:-2] + (-1,)).any(axis=-1)
    near = (mism & by_cut).reshape(switch.shape + (-1,)).any(axis=-1)
    worst = 0.0
    strict = np.zeros(switch.shape, dtype=bool)
    floor_needed = np.zeros(switch.shape, dtype=bool)
    for v in range(nv):
        b = Fo[v]
        a = Fg[v]
        err = np.where(switch, 0.0, np.abs(a - b))
        den0 = np.abs(b)
        fl_v = 1e-3 * np.max(np.abs(b)) + 1e-300
        den = np.maximum(den0, fl_v) if scale is None else np.maximum(den0, scale[v])
        if floor and scale is not None:
            den = np.maximum(den, fl_v)
        r = err / np.maximum(den, 1e-300)
        m = float(r.max())
        if m > rel:
            i = np.unravel_index(np.argmax(r), r.shape)
            raise AssertionError("%s: component %d face %s rel err %.3e (gpu %.17g oracle %.17g%s)"
                                 % (label, v, i, m, a[i], b[i],
                                    "" if scale is None else ", terms %.3e" % scale[v][i]))
        worst = max(worst, m)
        strict |= err > rel * den0
        if scale is not None:
            floor_needed |= err > rel * np.maximum(den0, scale[v])
    stats = {"switch_faces": int(switch.sum()), "near_cutoff_faces": int(near.sum()),
             "noise_faces": int((switch & ~near).sum()), "faces": int(switch.size), "max_rel": worst,
             "flag_mismatch": int(mism.sum()), "strict_faces": int(strict.sum()),
             "floor_faces": int(floor_needed.sum())}
    _log(label, stats)
    return stats


def bound_counts(st, noise_frac=0.01, floor=False):
    """The excused counts stay small: near-cutoff and noise-decided switch faces, each at
    most a fraction of the faces (at least 2); no face needs the 1e-3 max|b| floor unless
    the comparison allowed it."""
    lim_n = max(2, noise_frac * st["faces"])
    assert st["near_cutoff_faces"] <= lim_n, st
    assert st["noise_faces"] <= lim_n, st
    if not floor:
        assert st["floor_faces"] == 0, st


def compare_rhs(rg, ro, Fo_list, dx, exclude=None, rel=1e-12, label=""):
    """Cell operator values: |a - b| <= rel * sum_a max|F_a,v| / dx_a per component."""
    nv = ro.shape[0]
    for v in range(nv):
        scale = sum(np.max(np.abs(F[v])) / d for F, d in zip(Fo_list, dx))
        err = np.abs(rg[v] - ro[v])
        if exclude is not None:
            err = np.where(exclude, 0.0, err)
        m = float(err.max()) / scale
        if m > rel:
            i = np.unravel_index(np.argmax(err), err.shape)
            raise AssertionError("%s: component %d cell %s err %.3e of scale (gpu %.17g oracle %.17g)"
                                 % (label, v, i, m, rg[v][i], ro[v][i]))


def switch_cells(switch_faces_per_axis, cell_shape):
    """Cells adjacent to a switch face on any axis (numpy (z, y, x) shapes)."""
    ex = np.zeros(cell_shape, dtype=bool)
    nd = len(cell_shape)
    for a, sw in enumerate(switch_faces_per_axis):
        ax = nd - 1 - a  # numpy axis of physical axis a
        lo = [slice(None)] * nd
        hi = [slice(None)] * nd
        lo[ax] = slice(0, -1)   # face i -> cell i (right neighbour)
        hi[ax] = slice(1, None)  # face i+1 -> cell i (left neighbour)
        ex |= sw[tuple(lo)] | sw[tuple(hi)]
    return ex


def dilate(mask, r):
    """Box dilation by r cells along every axis, with periodic wrap (the cells whose
    values a switch at one of mask's cells can reach through r stencil half-widths)."""
    out = mask.copy()
    for ax in range(mask.ndim):
        cur = out.copy()
        for k in range(1, r + 1):
            cur |= np.roll(out, k, axis=ax) | np.roll(out, -k, axis=ax)
        out = cur
    return out


def compare_cells(Ug, Uo, exclude=None, rel=1e-13, label=""):
    """State values cell by cell: |a - b| <= rel * max(|b|, 1e-3 max|b|) per component
    (the floor for components that cross zero, e.g. momentum), outside `exclude`."""
    worst = 0.0
    for v in range(Uo.shape[0]):
        b, a = Uo[v], Ug[v]
        den = np.maximum(np.abs(b), 1e-3 * np.max(np.abs(b)) + 1e-300)
        r = np.abs(a - b) / den
        if exclude is not None:
            r = np.where(exclude, 0.0, r)
        m = float(r.max())
        if m > rel:
            i = np.unravel_index(np.argmax(r), r.shape)
            raise AssertionError("%s: component %d cell %s rel err %.3e (gpu %.17g oracle %.17g)"
                                 % (label, v, i, m, a[i], b[i]))
        worst = max(worst, m)
    return worst


CENTRAL = {6: np.array([1, -8, 37, 37, -8, 1]) / 60.0,
           8: np.array([-3, 29, -139, 533, 533, -139, 29, -3]) / 840.0}


def central_terms(U, axis, K, bc, gamma=1.4):
    """sum_q |c_q| |F_axis(U_{f-K/2+q})| per component and face of `axis` (x-first axis
    index; U numpy [nv, (nz,) (ny,) nx]; bc 0 periodic, 1 zero-gradient): the magnitude of
    the terms of the face's K-point central flux.  Returns [nv, face shape]."""
    nv = U.shape[0]
    nd = nv - 2
    rho = U[0]
    vel = [U[1 + d] / rho for d in range(nd)]
    p = (gamma - 1.0) * (U[nv - 1] - 0.5 * sum(U[1 + d] * vel[d] for d in range(nd)))
    un = vel[axis]
    F = [U[0] * un] + [U[1 + d] * un + (p if d == axis else 0.0) for d in range(nd)] + [(U[nv - 1] + p) * un]
    A = np.abs(np.stack(F))
    ax = 1 + (nd - 1 - axis)  # numpy axis of the sweep axis in [nv, ...]
    H = K // 2
    pad = [(0, 0)] * A.ndim
    pad[ax] = (H, H)
    Ap = np.pad(A, pad, mode="wrap" if bc == 0 else "edge")
    n = A.shape[ax]
    out = 0.0
    for q, cq in enumerate(CENTRAL[K]):
        sl = [slice(None)] * A.ndim
        sl[ax] = slice(q, q + n + 1)  # face f: cell f - H + q = padded index f + q
        out = out + abs(cq) * Ap[tuple(sl)]
    return out


def central_terms_at(U, axis, K, bc, idx, gamma=1.4):
    """central_terms at selected faces: idx[m, 3] = (x, y, z), the face index on `axis`.
    Returns [nv, m]."""
    nv = U.shape[0]
    nd = nv - 2
    n = U.shape[1:][::-1]  # (nx, ny, nz)
    H = K // 2
    out = np.zeros((nv, idx.shape[0]))
    for q, cq in enumerate(CENTRAL[K]):
        cell = idx[:, :nd].astype(np.int64).copy()
        j = cell[:, axis] - H + q
        j = np.mod(j, n[axis]) if bc == 0 else np.clip(j, 0, n[axis] - 1)
        cell[:, axis] = j
        sel = tuple(cell[:, d] for d in reversed(range(nd)))
        u = np.stack([U[v][sel] for v in range(nv)])
        rho = u[0]
        vel = [u[1 + d] / rho for d in range(nd)]
        p = (gamma - 1.0) * (u[nv - 1] - 0.5 * sum(u[1 + d] * vel[d] for d in range(nd)))
        un = vel[axis]
        F = [u[0] * un] + [u[1 + d] * un + (p if d == axis else 0.0) for d in range(nd)] + [(u[nv - 1] + p) * un]
        out += abs(cq) * np.abs(np.stack(F))
    return out
