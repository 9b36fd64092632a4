"""Parity metric of the GPU path against the oracle.

For each variable q: max |q_gpu - q_oracle| / scale, where the scale is the largest
magnitude over the variable's physical field in the oracle result: rho and p on
their own, the three velocity components together (the speed), the three field
components together, D, the three momentum components together, U.  Normalising
a vector component by the magnitude of its vector keeps components that are zero
or small by cancellation (v_x of a wave along y, say) well defined.  The bar for
FP64 is 1e-10 on smooth problems.
"""
import numpy as np

FP64_TOL = 1e-10

PRIM_GROUPS = [[0], [1, 2, 3], [4], [5, 6, 7]]       # rho | v | p | B
CONS_GROUPS = [[0], [1, 2, 3], [4]]                   # D | S | U
FACE_GROUPS = [[0, 1, 2]]                             # face B (or dB/dt)


def rel_errors(got, ref, groups, floor=1e-300):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    out = np.zeros(ref.shape[0])
    for grp in groups:
        scale = max(np.max(np.abs(ref[grp])), floor)
        if grp[-1] >= ref.shape[0]:
            raise IndexError("group %s out of range" % grp)
        for v in grp:
            out[v] = np.max(np.abs(got[v] - ref[v])) / scale
    return out


def assert_parity(got, ref, groups, tol=FP64_TOL, what="", floor=1e-300):
    e = rel_errors(got, ref, groups, floor)
    assert np.all(e <= tol), "%s parity errors %s > %g" % (what, np.array2string(e), tol)
    return e
