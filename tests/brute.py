"""Dense-matrix formulation of one explicit step (test helper, small grids only).

Independent of the oracle's stencil loops: the step is written as
theta' = A theta + c with A assembled entry by entry from the grid's
neighbour relation, so that theta^N = A^N theta^0 + sum_{k<N} A^k c can be
formed by repeated squaring of the augmented matrix [[A, c], [0, 1]].
"""
import numpy as np


def neighbours(nx, ny, nz, x, y, z):
    for dx, dy, dz in ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)):
        X, Y, Z = x + dx, y + dy, z + dz
        if 0 <= X < nx and 0 <= Y < ny and 0 <= Z < nz:
            yield X, Y, Z


def step_matrix(a, b, c_src, isfixed):
    """A and c of one step; a, b, c_src, isfixed are [nz, ny, nx] arrays."""
    nz, ny, nx = a.shape
    n = nx * ny * nz
    A = np.zeros((n, n))
    c = np.zeros(n)
    lin = lambda x, y, z: (z * ny + y) * nx + x
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                j = lin(x, y, z)
                if isfixed[z, y, x]:
                    A[j, j] = 1.0
                    continue
                nb = list(neighbours(nx, ny, nz, x, y, z))
                A[j, j] = 1.0 - a[z, y, x] * len(nb) - b[z, y, x]
                for (X, Y, Z) in nb:
                    A[j, lin(X, Y, Z)] += a[z, y, x]
                c[j] = c_src[z, y, x]
    return A, c


def power_augmented(A, c, N):
    n = A.shape[0]
    M = np.zeros((n + 1, n + 1))
    M[:n, :n] = A
    M[:n, n] = c
    M[n, n] = 1.0
    return np.linalg.matrix_power(M, N)


def evolve(A, c, theta0, N):
    MN = power_augmented(A, c, N)
    n = A.shape[0]
    return MN[:n, :n] @ theta0 + MN[:n, n]


def step_matrix_faces(wf, b, c_src, isfixed):
    """A and c of one step of the conservative form: free voxel j gets weight
    wf[d][j] on its neighbour in direction d (x-, x+, y-, y+, z-, z+) and
    1 - sum_d wf[d][j] - b[j] on itself."""
    nz, ny, nx = b.shape
    n = nx * ny * nz
    A = np.zeros((n, n))
    c = np.zeros(n)
    lin = lambda x, y, z: (z * ny + y) * nx + x
    offs = ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1))
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                j = lin(x, y, z)
                if isfixed[z, y, x]:
                    A[j, j] = 1.0
                    continue
                diag = 1.0 - b[z, y, x]
                for d, (dx, dy, dz) in enumerate(offs):
                    X, Y, Z = x + dx, y + dy, z + dz
                    if 0 <= X < nx and 0 <= Y < ny and 0 <= Z < nz:
                        A[j, lin(X, Y, Z)] += wf[d, z, y, x]
                        diag -= wf[d, z, y, x]
                A[j, j] = diag
                c[j] = c_src[z, y, x]
    return A, c
