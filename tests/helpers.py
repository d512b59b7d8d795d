"""Shared comparison helpers for the parity tests."""
import numpy as np

# The trend tolerance is 1e-5 relative per sample.  For curves centred near
# zero (synthetic edge cases, not flux) a relative bound is meaningless, so
# those use 1e-5 of max(|trend|, c * s): the FP32 path's error scales with
# the window's spread (c s) as well as with the level.
TREND_RTOL = 1e-5


def compare_diag(got, ref, c=5.0, scale_aware=False, what="", x=None):
    """got: dict of numpy arrays from the GPU diag path; ref: oracle dict."""
    n = ref["trend"].size
    assert got["trend"].size == n
    # Counts are integers: bit-exact.
    np.testing.assert_array_equal(got["nvalid"], ref["nvalid"], err_msg=what + " nvalid")
    np.testing.assert_array_equal(got["nplus"], ref["nplus"], err_msg=what + " nplus")
    # Median: an FP32 order statistic of the inputs, compared as a value.
    mref = ref["median"]
    mgot = got["median"].astype(np.float64)
    np.testing.assert_array_equal(np.isnan(mgot), np.isnan(mref), err_msg=what + " median NaN")
    ok = ~np.isnan(mref)
    bad = np.nonzero(mgot[ok] != mref[ok])[0]
    assert bad.size == 0, "%s median differs at %s: %s vs %s" % (
        what, np.nonzero(ok)[0][bad[:5]], mgot[ok][bad[:5]], mref[ok][bad[:5]])
    compare_trend(got["trend"], ref["trend"], ref.get("scale"), c, scale_aware, what)
    if scale_aware:
        # x / trend amplifies the trend's error by |x| / trend^2 where the trend
        # is near zero; check the NaN pattern and that detr is the IEEE
        # quotient of the sample by the GPU's own trend instead.
        np.testing.assert_array_equal(np.isnan(got["detr"]), np.isnan(ref["detr"]),
                                      err_msg=what + " detr NaN pattern")
        if x is not None:
            ok = ~np.isnan(ref["detr"])
            with np.errstate(divide="ignore", invalid="ignore"):   # a zero trend gives +-inf
                q = (x[ok].astype(np.float32) / got["trend"][ok].astype(np.float32))
            np.testing.assert_array_equal(got["detr"][ok], q, err_msg=what + " detr quotient")
    else:
        compare_detr(got["detr"], ref["detr"], what)


def compare_trend(tgot, tref, sref=None, c=5.0, scale_aware=False, what=""):
    tgot = np.asarray(tgot, np.float64)
    np.testing.assert_array_equal(np.isnan(tgot), np.isnan(tref), err_msg=what + " trend NaN pattern")
    ok = ~np.isnan(tref)
    if not ok.any():
        return
    bound = np.abs(tref[ok])
    if scale_aware and sref is not None:
        bound = np.maximum(bound, c * np.nan_to_num(sref[ok]))
    err = np.abs(tgot[ok] - tref[ok])
    lim = TREND_RTOL * bound
    worst = np.argmax(err - lim)
    assert np.all(err <= lim), "%s trend off at %d: got %r ref %r (err %g, lim %g)" % (
        what, np.nonzero(ok)[0][worst], tgot[ok][worst], tref[ok][worst], err[worst], lim[worst])


def compare_detr(dgot, dref, what=""):
    dgot = np.asarray(dgot, np.float64)
    np.testing.assert_array_equal(np.isnan(dgot), np.isnan(dref), err_msg=what + " detr NaN pattern")
    ok = ~np.isnan(dref) & np.isfinite(dref)
    err = np.abs(dgot[ok] - dref[ok])
    lim = TREND_RTOL * np.abs(dref[ok]) + 1e-30
    assert np.all(err <= lim), "%s detr off by %g" % (what, float((err / lim).max()))


def depth_recovery_errors(detr, batch, idx=None):
    """Per-curve absolute percentage depth errors; the measure is the
    package's (paper_2604_06602_gb300.injection.depth_errors)."""
    from paper_2604_06602_gb300.injection import depth_errors
    return depth_errors(detr, batch, idx)
