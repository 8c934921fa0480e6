"""Test helpers: layout conversions and dense assembly (no simulator arithmetic)."""
import numpy as np

# neighbour offsets of the 7-point stencil: centre, -x, +x, -y, +y, -z, +z
DIRS = [(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]


def neighbour(nx, ny, nz, i, d):
    ix, iy, iz = i % nx, (i // nx) % ny, i // (nx * ny)
    dx, dy, dz = DIRS[d]
    jx, jy, jz = ix + dx, iy + dy, iz + dz
    if 0 <= jx < nx and 0 <= jy < ny and 0 <= jz < nz:
        return jx + nx * (jy + ny * jz)
    return -1


def dense_from_blocks(J, nx, ny, nz):
    """Dense (N b) x (N b) matrix from oracle-layout blocks J[i, d, r, c]."""
    N, _, b, _ = J.shape
    A = np.zeros((N * b, N * b))
    for i in range(N):
        for d in range(7):
            j = neighbour(nx, ny, nz, i, d)
            if j >= 0:
                A[i * b:(i + 1) * b, j * b:(j + 1) * b] += J[i, d]
    return A


def cell_major(v, N, b):
    """[b][N] component-major vector -> interleaved [N][b]."""
    return np.asarray(v).reshape(b, N).T.reshape(-1)


def comp_major(v, N, b):
    """interleaved [N][b] -> [b][N] component-major."""
    return np.asarray(v).reshape(N, b).T.reshape(-1)


def random_state(case, seed, N, b):
    """A random but physical iterate, both phase states for black oil."""
    rng = np.random.default_rng(seed)
    x = np.zeros((N, b))
    x[:, 0] = case["init"]["p"] + rng.uniform(-20, 20, N)
    x[:, 1] = rng.uniform(0.12, 0.55, N)
    ph = np.ones(N, np.int8)
    if b == 3:
        ph = (rng.uniform(size=N) < 0.5).astype(np.int8)
        x[:, 2] = np.where(ph == 1, rng.uniform(0.06, 0.25, N), x[:, 0] - rng.uniform(5, 40, N))
    return x.reshape(-1), ph
