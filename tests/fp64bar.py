"""The FP64 parity bar shared by the GPU tests (test helper, no fixtures).

|gpu - oracle| <= 1e-12 * absum on every CSR entry, where absum is the
oracle's sum of the magnitudes of the entry's expanded quadrature terms
(Section 3, step 4: every entry is a quadrature sum), so that an entry which
cancels is judged against the size of what cancelled; and, on the entries
that do not cancel (|oracle| >= 1e-3 * absum), the plain relative error
|gpu - oracle| / |oracle| <= 1e-12.
"""
import numpy as np

FP64_TOL = 1e-12


def check_fp64(g, o, absum, what=""):
    """Asserts both parts of the bar; returns (worst error / bound on the
    absum part, worst plain relative error on the non-cancelling entries)."""
    g, o, absum = (np.asarray(x, dtype=np.float64) for x in (g, o, absum))
    err = np.abs(g - o)
    worst_abs = float((err / (FP64_TOL * absum + 1e-300)).max()) if err.size else 0.0
    assert worst_abs <= 1.0, (what, "per entry vs absum", worst_abs)
    big = (np.abs(o) >= 1e-3 * absum) & (absum > 0)
    worst_rel = float((err[big] / np.abs(o[big])).max()) if big.any() else 0.0
    assert worst_rel <= FP64_TOL, (what, "plain relative", worst_rel)
    return worst_abs, worst_rel
