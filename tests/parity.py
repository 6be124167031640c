"""Parity rules between the CUDA path and the CPU oracle (test-side helper).

Face values: |a - b| <= REL * max(|b|, 1e-3 * max_faces |b| of that component, S) where S is
the magnitude of the terms of the characteristic back-projection sum_s r_s (f+_s + f-_s)
that forms the face value (reported by the oracle): a face value that is small because
those terms cancel is measured against the terms, as for any floating-point sum.
Flags (delta_k bits and the adaptive C_T code): identical, except where the oracle's
decision is ill-conditioned in FP64 -- its chi_k (or the adaptive beta) lies within
CUT_TOL relative of the threshold, or within NOISE_K times the sequence's rounding-noise
ratio (a characteristic sequence that is constant up to rounding, e.g. the acoustic
fields across a contact, has indicators made of rounding noise).  Faces with such a
mismatch ("switch faces") are counted and excluded from the value check.
"""
import numpy as np

REL = 1e-13
CUT_TOL = 1e-10
NOISE_K = 1e4


def compare_faces(Fg, flg, Fo, flo, cut, noise, scale=None, rel=REL, label=""):
    """Fg/Fo/scale: [nv, *faces]; flg/flo/cut/noise: [*faces, nv, 2].  Returns a stats dict;
    raises AssertionError on a violation."""
    nv = Fo.shape[0]
    mism = flg != flo
    allowed = (cut <= CUT_TOL) | (cut <= NOISE_K * noise)
    bad = mism & ~allowed
    n_bad = int(bad.sum())
    if n_bad:
        idx = np.argwhere(bad)[:5]
        info = [(tuple(i), int(flg[tuple(i)]), int(flo[tuple(i)]), float(cut[tuple(i)]), float(noise[tuple(i)]))
                for i in idx]
        raise AssertionError("%s: %d flag mismatches away from the cutoff, e.g. %s" % (label, n_bad, info))
    # faces whose flags legitimately differ are excluded from the value check
    switch = mism.reshape(mism.shape[:-2] + (-1,)).any(axis=-1)
    near = (mism & (cut <= CUT_TOL)).reshape(switch.shape + (-1,)).any(axis=-1)
    worst = 0.0
    for v in range(nv):
        b = Fo[v]
        a = Fg[v]
        den = np.maximum(np.abs(b), 1e-3 * np.max(np.abs(b)) + 1e-300)
        if scale is not None:
            den = np.maximum(den, scale[v])
        r = np.abs(a - b) / den
        r = np.where(switch, 0.0, r)
        m = float(r.max())
        if m > rel:
            i = np.unravel_index(np.argmax(r), r.shape)
            raise AssertionError("%s: component %d face %s rel err %.3e (gpu %.17g oracle %.17g)"
                                 % (label, v, i, m, a[i], b[i]))
        worst = max(worst, m)
    return {"switch_faces": int(switch.sum()), "near_cutoff_faces": int(near.sum()),
            "noise_faces": int((switch & ~near).sum()), "faces": int(switch.size), "max_rel": worst,
            "flag_mismatch": int(mism.sum())}


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
