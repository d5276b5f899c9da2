"""The FP64 parity bar shared by the GPU tests (test helper, no fixtures).

|gpu - oracle| <= 1e-12 * absum on every CSR entry, where absum is the
oracle's sum of the magnitudes of the entry's expanded quadrature terms
(Section 3, step 4: every entry is a quadrature sum), so that an entry which
cancels is judged against the size of what cancelled.  On the entries that
do not cancel, the plain relative error |gpu - oracle| / |oracle| is bounded
too: by 1e-12 where |oracle| >= 0.1 absum, and by 1e-10 where
|oracle| >= 1e-3 absum.  (Both sides carry rounding errors of a few units
of 2^-53 times absum, times the number of terms, up to ~100 units for the
P3 mass-tensor term; an entry at 1e-3 absum reads that as up to ~2e-11
relative, which the absum bar alone would let grow to 1e-9.)
"""
import numpy as np

FP64_TOL = 1e-12


def check_fp64(g, o, absum, what="", rel_factor=1.0):
    """Asserts the bar; returns (worst error / bound on the absum part,
    worst plain relative error where |o| >= 0.1 absum, worst where
    |o| >= 1e-3 absum).  rel_factor widens the two plain relative tiers
    (not the absum bar) for quantities whose terms are products of three
    basis functions (the mass tensor of Section 5.1), which amplify the
    1e-14 moment residuals of the library's numerically derived
    quadrature rules."""
    g, o, absum = (np.asarray(x, dtype=np.float64) for x in (g, o, absum))
    err = np.abs(g - o)
    worst_abs = float((err / (FP64_TOL * absum + 1e-300)).max()) if err.size else 0.0
    assert worst_abs <= 1.0, (what, "per entry vs absum", worst_abs)
    out = [worst_abs]
    for frac, tol in ((0.1, rel_factor * FP64_TOL), (1e-3, rel_factor * 100 * FP64_TOL)):
        big = (np.abs(o) >= frac * absum) & (absum > 0)
        worst = float((err[big] / np.abs(o[big])).max()) if big.any() else 0.0
        assert worst <= tol, (what, f"plain relative where |o| >= {frac} absum", worst)
        out.append(worst)
    return tuple(out)
