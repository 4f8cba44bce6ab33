"""Textbook lattice constants and a vectorised plain-LBGK step written in
numpy, used by the tests as an independent check of the oracle's fluid part
(no particles: the beta -> 0 limit of Eq. 1)."""
import numpy as np

# direction order of the library interface: rest, then +-pairs
D2Q9_C = np.array([[0, 0], [1, 0], [-1, 0], [0, 1], [0, -1], [1, 1], [-1, -1], [1, -1], [-1, 1]])
D2Q9_W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
D3Q19_C = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                    [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1], [1, 0, -1],
                    [-1, 0, 1], [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]])
D3Q19_W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def lattice(dim):
    if dim == 2:
        c = np.zeros((9, 3), dtype=int)
        c[:, :2] = D2Q9_C
        return c, D2Q9_W
    return D3Q19_C.copy(), D3Q19_W


def opposite(c):
    return np.array([int(np.nonzero((c == -ci).all(axis=1))[0][0]) for ci in c])


def numpy_lbgk_step(f, dim, tau, g, wall_y):
    """f: post-collision populations (Q, nz, ny, nx).  Returns the next
    post-collision populations: pull streaming (np.roll on the periodic axes,
    halfway bounce-back at y walls), BGK relaxation, F_i = 3 w_i rho c_i.g."""
    c, w = lattice(dim)
    opp = opposite(c)
    Q = len(w)
    ft = np.empty_like(f)
    for i in range(Q):
        # f~_i(x) = f*_i(x - c_i): roll by +c_i (axes: z=1, y=2, x=3)
        ft[i] = np.roll(f[i], shift=(c[i, 2], c[i, 1], c[i, 0]), axis=(0, 1, 2))
        if wall_y and c[i, 1] != 0:
            ny = f.shape[2]
            rows = [0] if c[i, 1] > 0 else [ny - 1]
            for y in rows:
                ft[i][:, y, :] = f[opp[i]][:, y, :]
    rho = ft.sum(axis=0)
    j = np.einsum("qd,qzyx->dzyx", c.astype(float), ft)
    u = j / rho
    uu = (u * u).sum(axis=0)
    out = np.empty_like(f)
    for i in range(Q):
        cu = c[i, 0] * u[0] + c[i, 1] * u[1] + c[i, 2] * u[2]
        feq = w[i] * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uu)
        Fi = 3 * w[i] * rho * (c[i] @ np.asarray(g, dtype=float))
        out[i] = ft[i] - (ft[i] - feq) / tau + Fi
    return out
