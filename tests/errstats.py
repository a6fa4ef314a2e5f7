"""Force-error measures of the parity tests: the relative RMS over an i-set,
sqrt(sum_i |d_i|^2 / sum_i |ref_i|^2), and the per-particle relative error |d_i| / |ref_i|
(its maximum and median over the set) for a vector (rows = particles) or scalar quantity."""
import numpy as np


def rel_rms(got, ref):
    ref = np.asarray(ref, dtype=np.float64)
    den = float((ref ** 2).sum())
    num = float(((np.asarray(got, dtype=np.float64) - ref) ** 2).sum())
    return np.sqrt(num / den) if den > 0 else np.sqrt(num)


def per_particle(got, ref):
    """(max, median) over the particles of |got_i - ref_i| / |ref_i|; rows are particles."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if ref.ndim == 1:
        d, r = np.abs(got - ref), np.abs(ref)
    else:
        d, r = np.linalg.norm(got - ref, axis=1), np.linalg.norm(ref, axis=1)
    keep = r > 0
    if not keep.any():
        return float(d.max()), float(np.median(d))
    e = d[keep] / r[keep]
    return float(e.max()), float(np.median(e))


def report(pairs):
    """{name: (rel_rms, max, median)} for pairs {name: (got, ref)}."""
    out = {}
    for name, (got, ref) in pairs.items():
        mx, med = per_particle(got, ref)
        out[name] = (rel_rms(got, ref), mx, med)
    return out


def fmt(rep):
    return "  ".join("%s rms %.2e max %.2e med %.2e" % (k, *v) for k, v in rep.items())
