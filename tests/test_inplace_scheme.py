"""The slot mapping of the in-place (AA) step, checked on the CPU with numpy.

A cell reads its 27 populations from slots s_q and writes its post-collision
f*_q to s_qbar: on even steps s_q is the pull source A[q][x - c_q] (wrapped on
periodic axes, A[qbar][x] past a no-slip wall), on odd steps s_q = A[qbar][x].
With any per-cell update (here a fixed random 27x27 mixing, which tells every
direction apart), an even and an odd step from the two-array state reproduce
two steps of the pull scheme exactly, and every step writes each slot once.
This is the mapping the CUDA kernel implements; the GPU tests compare the
kernel itself with the pull scheme bitwise."""
import itertools

import numpy as np
import pytest

C = np.array([[q % 3 - 1, (q // 3) % 3 - 1, q // 9 - 1] for q in range(27)])


def _src(shape, bc, x, y, z, c):
    """Source cell of a pull along c, or None past a no-slip wall."""
    s = [x - c[0], y - c[1], z - c[2]]
    for a, n in enumerate(shape):
        if not 0 <= s[a] < n:
            if bc[a] != "periodic":
                return None
            s[a] %= n
    return tuple(s)


def _pull_step(A, shape, bc, M):
    nx, ny, nz = shape
    B = np.empty_like(A)
    for x, y, z in itertools.product(range(nx), range(ny), range(nz)):
        h = np.empty(27)
        for q in range(27):
            s = _src(shape, bc, x, y, z, C[q])
            h[q] = A[26 - q, z, y, x] if s is None else A[q, s[2], s[1], s[0]]
        B[:, z, y, x] = M @ h
    return B


def _aa_step(A, shape, bc, M, odd, writes):
    nx, ny, nz = shape
    for x, y, z in itertools.product(range(nx), range(ny), range(nz)):
        slots = []
        for q in range(27):
            if odd:
                slots.append((26 - q, z, y, x))
            else:
                s = _src(shape, bc, x, y, z, C[q])
                slots.append((26 - q, z, y, x) if s is None else (q, s[2], s[1], s[0]))
        h = np.array([A[sl] for sl in slots])
        out = M @ h
        for q in range(27):
            A[slots[26 - q]] = out[q]
            writes[slots[26 - q]] += 1


@pytest.mark.parametrize("shape,bc", [((5, 4, 3), ("periodic",) * 3),
                                      ((4, 5, 3), ("noslip", "periodic", "noslip")),
                                      ((3, 3, 4), ("noslip",) * 3),
                                      ((1, 4, 2), ("periodic", "noslip", "periodic"))])
def test_even_and_odd_steps_reproduce_the_pull_scheme(shape, bc):
    rng = np.random.default_rng(5)
    nx, ny, nz = shape
    M = rng.normal(size=(27, 27))
    A0 = rng.normal(size=(27, nz, ny, nx))
    ref = _pull_step(_pull_step(A0, shape, bc, M), shape, bc, M)
    A = A0.copy()
    for odd in (False, True):
        writes = np.zeros(A.shape, dtype=int)
        _aa_step(A, shape, bc, M, odd, writes)
        assert np.all(writes == 1)          # every slot written exactly once per step
    np.testing.assert_allclose(A, ref, rtol=0, atol=1e-12)
