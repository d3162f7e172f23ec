"""Layout helpers shared by the tests (no method arithmetic)."""
import numpy as np


def unpack_rho(packed, D):
    """vec_h (..., D*D) -> complex (..., D, D): Re rho_ii on the diagonal, Re rho_ij above
    it, Im rho_ij below it (the layout documented in include/qst.h)."""
    a = np.asarray(packed, dtype=np.float64).reshape(*np.shape(packed)[:-1], D, D)
    upper = np.triu(np.ones((D, D), bool), 1)
    at = np.swapaxes(a, -1, -2)
    diag = np.diagonal(a, axis1=-2, axis2=-1)[..., None] * np.eye(D)
    re = np.where(upper, a, 0.0) + np.where(upper.T, at, 0.0) + diag
    im_upper = np.where(upper, -at, 0.0)
    im = im_upper - np.swapaxes(im_upper, -1, -2)
    return re + 1j * im


def pack_rho(rho):
    """complex (..., D, D) -> vec_h (..., D*D), inverse of unpack_rho."""
    rho = np.asarray(rho)
    D = rho.shape[-1]
    upper = np.triu(np.ones((D, D), bool), 1)
    out = np.where(upper, rho.real, 0.0) + np.where(upper.T, rho.imag, 0.0) + \
        np.diagonal(rho.real, axis1=-2, axis2=-1)[..., None] * np.eye(D)
    return out.reshape(*rho.shape[:-2], D * D)


def near_tie_band(acc_gpu, acc_ref, ll_prop_gpu, ll_prop_ref):
    """Band within which an accept decision may legitimately differ from the oracle's: twice
    the largest |log L(y') GPU - oracle| measured in the same run (the current and the
    proposed state each carry one error), over every chain-step up to and including a
    chain's first differing decision (until then both sides hold identical states), finite
    entries only.  Arrays are [chains, steps]."""
    acc_gpu = np.asarray(acc_gpu)
    acc_ref = np.asarray(acc_ref)
    R, S = acc_ref.shape
    first = np.full(R, S)
    for r in range(R):
        bad = np.nonzero(acc_gpu[r] != acc_ref[r])[0]
        if bad.size:
            first[r] = bad[0] + 1
    mask = np.arange(S)[None, :] < first[:, None]
    a = np.asarray(ll_prop_gpu, dtype=np.float64)
    b = np.asarray(ll_prop_ref, dtype=np.float64)
    ok = mask & np.isfinite(a) & np.isfinite(b)
    return 2.0 * np.abs(a[ok] - b[ok]).max() + 1e-9
