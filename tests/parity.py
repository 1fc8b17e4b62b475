"""Helpers shared by the GPU parity tests: move a GPU state into the oracle
and build the comparison masks of the stated tolerances."""
import numpy as np
from scipy import ndimage

from oracle import lsgg_oracle as O


def oracle_from_gpu(shape_zyx, boxes, phi_by_grain, idf_by_grain=None, physics=None):
    """Oracle microstructure holding exactly the GPU's FP32 state (as FP64)."""
    grains = []
    for g, b in enumerate(boxes):
        if b[0]:
            gr = O.Grain(g, (int(b[3]), int(b[2]), int(b[1])), phi_by_grain[g].astype(np.float64))
            if idf_by_grain is not None:
                gr.idf = idf_by_grain[g].astype(np.int64)
            grains.append(gr)
        else:
            grains.append(O.Grain(g, (0, 0, 0), np.full((1, 1, 1), -7.0), alive=False))
    return O.Microstructure(tuple(shape_zyx), grains, physics=physics)


def sign_flip_exclusion(ref_c, gpu_c, full, tol=1e-4, reach=7):
    """Cells to skip: within `reach` taxicab steps of a cell where the oracle
    and the GPU disagree on the sign of phi_c and |phi_c| < tol."""
    bad = ((ref_c > 0) != (gpu_c > 0)) & (np.abs(ref_c) < tol)
    if not bad.any():
        return np.zeros(ref_c.shape, bool)
    st = ndimage.generate_binary_structure(ref_c.ndim, 1)
    if ref_c.shape[0] == 1:
        st[0] = False
        st[2] = False
        st[1, 1, 1] = True
    out = bad.copy()
    for _ in range(reach):
        grown = ndimage.binary_dilation(out, structure=st)
        # periodic wrap on full axes
        for ax in range(3):
            if full[ax] and ref_c.shape[ax] > 1:
                grown |= np.roll(out, 1, axis=ax) | np.roll(out, -1, axis=ax)
        out = grown
    return out


def box_full(b, shape_zyx):
    return (b[6] == shape_zyx[0], b[5] == shape_zyx[1], b[4] == shape_zyx[2])
