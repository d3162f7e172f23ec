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
