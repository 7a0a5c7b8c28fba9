"""Independent dense-array formulations of the periodic level operators, used
to pin the oracle (which works on octs, Morton keys and hash lookups).

Nothing here shares code with the oracle or the CUDA library: these are the
textbook 7-point operators on an n^3 periodic array indexed a[x, y, z], written
with np.roll.  Cell (x, y, z) is red when x + y + z is even (App. D.2 update,
red first)."""
import numpy as np


def nb_sum(phi):
    s = np.roll(phi, 1, 0)
    s = s + np.roll(phi, -1, 0)
    s = s + np.roll(phi, 1, 1)
    s = s + np.roll(phi, -1, 1)
    s = s + np.roll(phi, 1, 2)
    s = s + np.roll(phi, -1, 2)
    return s


def red_mask(n):
    x, y, z = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    return (x + y + z) % 2 == 0


def rb_sweep(phi, f, h):
    phi = phi.copy()
    red = red_mask(phi.shape[0])
    for mask in (red, ~red):
        new = (nb_sum(phi) - h * h * f) * (1.0 / 6.0)
        phi[mask] = new[mask]
    return phi


def laplacian(phi, h):
    return (nb_sum(phi) - 6.0 * phi) / (h * h)


def residual(phi, f, h):
    return f - laplacian(phi, h)


def restrict(r):
    n = r.shape[0] // 2
    return r.reshape(n, 2, n, 2, n, 2).mean(axis=(1, 3, 5))


def prolong(e):
    """Cell-centred trilinear interpolation of a periodic coarse array onto the
    fine cells: weights 3/4 (own coarse cell) and 1/4 (neighbour toward the
    fine cell) per axis."""
    n = e.shape[0]
    out = np.zeros((2 * n,) * 3)
    for px in (0, 1):
        for py in (0, 1):
            for pz in (0, 1):
                o = [1 if p else -1 for p in (px, py, pz)]
                acc = np.zeros_like(e)
                for cx in (0, 1):
                    for cy in (0, 1):
                        for cz in (0, 1):
                            w = (0.25 if cx else 0.75) * (0.25 if cy else 0.75) * (0.25 if cz else 0.75)
                            sh = (-o[0] * cx, -o[1] * cy, -o[2] * cz)
                            acc = acc + w * np.roll(e, sh, axis=(0, 1, 2))
                out[px::2, py::2, pz::2] = acc
    return out


def fft_solve(f, h):
    """Exact solution of the periodic 7-point problem L_h phi = f (zero mean):
    eigenvalues -(4/h^2) sum_d sin^2(pi k_d / n)."""
    n = f.shape[0]
    k = np.arange(n)
    s = np.sin(np.pi * k / n) ** 2
    lam = -(4.0 / (h * h)) * (s[:, None, None] + s[None, :, None] + s[None, None, :])
    fh = np.fft.fftn(f)
    lam[0, 0, 0] = 1.0
    ph = fh / lam
    ph[0, 0, 0] = 0.0
    return np.real(np.fft.ifftn(ph))


def dense_matrix(n, h):
    """The periodic 7-point operator as an explicit (n^3 x n^3) matrix."""
    N = n ** 3
    A = np.zeros((N, N))
    idx = np.arange(N).reshape(n, n, n)
    for x in range(n):
        for y in range(n):
            for z in range(n):
                i = idx[x, y, z]
                A[i, i] -= 6.0 / (h * h)
                for d in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    j = idx[(x + d[0]) % n, (y + d[1]) % n, (z + d[2]) % n]
                    A[i, j] += 1.0 / (h * h)
    return A
