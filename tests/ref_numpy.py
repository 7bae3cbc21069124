"""A second, independent FP64 form of Eq. 1 used only to cross-check the C
oracle: three tensor contractions with the dense n x n DFT matrix
M[j, k] = exp(s 2 pi i j k / n), built from NumPy's exp of the exact reduced
angle.  Never used on the product path."""
import numpy as np


def dft_matrix(n: int, sign: int) -> np.ndarray:
    j = np.arange(n)
    m = np.outer(j, j) % n
    return np.exp(sign * 2j * np.pi * m / n)


def dft3d_tensordot(x, sign: int = -1) -> np.ndarray:
    a = np.asarray(x, dtype=np.complex128)
    nz, ny, nx = a.shape[-3:]
    a = np.tensordot(a, dft_matrix(nx, sign), axes=([a.ndim - 1], [0]))       # x
    a = np.moveaxis(np.tensordot(a, dft_matrix(ny, sign), axes=([a.ndim - 2], [0])), -1, -2)  # y
    a = np.moveaxis(np.tensordot(a, dft_matrix(nz, sign), axes=([a.ndim - 3], [0])), -1, -3)  # z
    return a
