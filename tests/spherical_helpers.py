"""Real solid harmonics of s, p, d shells from Cartesian components, written
out for the tests (independently of the library's constants).

Cartesian order per shell: p = x, y, z; d = xx, xy, xz, yy, yz, zz, every
component carrying the normalisation of the axial x^l component.  The real
solid harmonics of a d shell, in the order xy, yz, z^2, xz, x^2 - y^2, are
sqrt3 xy, sqrt3 yz, (2zz - xx - yy)/2, sqrt3 xz and sqrt3/2 (xx - yy), which
are orthonormal in that normalisation (pinned by test_oracle_spherical)."""
import numpy as np

R3 = np.sqrt(3.0)
T_D = np.array([
    [0.0, R3, 0.0, 0.0, 0.0, 0.0],
    [0.0, 0.0, 0.0, 0.0, R3, 0.0],
    [-0.5, 0.0, 0.0, -0.5, 0.0, 1.0],
    [0.0, 0.0, R3, 0.0, 0.0, 0.0],
    [R3 / 2, 0.0, 0.0, -R3 / 2, 0.0, 0.0],
])


def shell_transform(l):
    return {0: np.eye(1), 1: np.eye(3), 2: T_D}[int(l)]


def system_transform(sysobj):
    """Block-diagonal T (n_sph x n_cart) of a system: phi_sph = T chi_cart."""
    blocks = [shell_transform(l) for l in sysobj.shell_l]
    n_s = sum(b.shape[0] for b in blocks)
    n_c = sum(b.shape[1] for b in blocks)
    T = np.zeros((n_s, n_c))
    r = c = 0
    for b in blocks:
        T[r:r + b.shape[0], c:c + b.shape[1]] = b
        r += b.shape[0]
        c += b.shape[1]
    return T


def spherical_K(K_cart_of, T, P_sph):
    """K in spherical harmonics of a spherical density: T K(T^T P T) T^T."""
    return T @ K_cart_of(T.T @ P_sph @ T) @ T.T
