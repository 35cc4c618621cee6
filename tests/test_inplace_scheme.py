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


# ---------------------------------------------------------------- every boundary rule

def _rule(shape, bc, x, y, z, q):
    """The pull rule of direction q at cell (x, y, z), in the order no-slip,
    free-slip, periodic wrap, x inlet / outlet.  Returns ("slot", (q', z, y, x)),
    ("ghost", (q', z, y)) for an inlet ghost population of column (y, z), or
    ("outlet", (q', z, y)) for the zero-gradient copy of the last plane."""
    n = shape
    c = list(C[q])
    p = [x, y, z]
    s = [p[a] - c[a] for a in range(3)]
    if any(bc[a] == "noslip" and not 0 <= s[a] < n[a] for a in range(3)):
        return "slot", (26 - q, z, y, x)
    cm = list(c)
    for a in range(3):
        if bc[a] == "freeslip" and not 0 <= s[a] < n[a]:
            cm[a] = -c[a]
            s[a] = p[a]
    for a in range(3):
        if bc[a] == "periodic":
            s[a] %= n[a]
    qm = (cm[2] + 1) * 9 + (cm[1] + 1) * 3 + (cm[0] + 1)
    if bc[0] == "inout" and s[0] < 0:
        return "ghost", (qm, s[2], s[1])
    if bc[0] == "inout" and s[0] >= n[0]:
        return "outlet", (qm, s[2], s[1])
    return "slot", (qm, s[2], s[1], s[0])


def _pull_step_full(A, shape, bc, M, G):
    nx, ny, nz = shape
    B = np.empty_like(A)
    for x, y, z in itertools.product(range(nx), range(ny), range(nz)):
        h = np.empty(27)
        for q in range(27):
            kind, key = _rule(shape, bc, x, y, z, q)
            if kind == "slot":
                h[q] = A[key]
            elif kind == "ghost":
                h[q] = G[key]
            else:                          # the clamp onto the last plane
                qm, zz, yy = key
                h[q] = A[qm, zz, yy, nx - 1]
        B[:, z, y, x] = M @ h
    return B


def _aa_step_full(A, shape, bc, M, G, OB, odd, writes):
    """One in-place step; OB holds the last plane's c_x = -1 populations of
    the previous step, and the step writes the next copy into a new buffer."""
    nx, ny, nz = shape
    OB_next = np.zeros_like(OB)
    for x, y, z in itertools.product(range(nx), range(ny), range(nz)):
        src = [_rule(shape, bc, x, y, z, q) for q in range(27)]
        h = np.empty(27)
        for q, (kind, key) in enumerate(src):
            if kind == "ghost":
                h[q] = G[key]
            elif kind == "outlet":
                h[q] = OB[key]
            else:
                h[q] = A[26 - q, z, y, x] if odd else A[key]
        out = M @ h
        if bc[0] == "inout" and x == nx - 1:
            for q in range(27):
                if C[q, 0] == -1:
                    OB_next[q, z, y] = out[q]
        for q in range(27):
            if odd:
                target = (q, z, y, x)
            else:
                kind, key = src[26 - q]    # the source read for the opposite direction
                if kind != "slot":
                    continue               # f*_q leaves the lattice
                target = key
            A[target] = out[q]
            writes[target] += 1
    return OB_next


@pytest.mark.parametrize("shape,bc", [((5, 4, 3), ("inout", "periodic", "periodic")),
                                      ((5, 4, 4), ("inout", "periodic", "freeslip")),
                                      ((4, 5, 3), ("freeslip", "noslip", "freeslip")),
                                      ((5, 3, 4), ("inout", "freeslip", "noslip")),
                                      ((3, 4, 4), ("periodic", "freeslip", "periodic")),
                                      ((1, 4, 3), ("periodic", "freeslip", "noslip"))])
def test_inplace_steps_with_inlet_outlet_and_free_slip_reproduce_the_pull_scheme(shape, bc):
    """With inlet ghosts, the outlet's zero-gradient copy kept in its own
    buffer, and free-slip mirrors, an even and an odd in-place step reproduce
    two pull steps exactly; no slot is written twice in a step, and after the
    odd step every slot has been written."""
    rng = np.random.default_rng(7)
    nx, ny, nz = shape
    M = rng.normal(size=(27, 27))
    A0 = rng.normal(size=(27, nz, ny, nx))
    Gs = [rng.normal(size=(27, nz, ny)) for _ in range(2)]   # ghost populations of steps 0 and 1
    ref = _pull_step_full(_pull_step_full(A0, shape, bc, M, Gs[0]), shape, bc, M, Gs[1])
    A = A0.copy()
    OB = np.zeros((27, nz, ny))
    for q in range(27):
        if C[q, 0] == -1:
            OB[q] = A0[q, :, :, nx - 1]                       # the copy taken at a state change
    for step, odd in ((0, False), (1, True)):
        writes = np.zeros(A.shape, dtype=int)
        OB = _aa_step_full(A, shape, bc, M, Gs[step], OB, odd, writes)
        assert writes.max() <= 1
        if odd:
            assert np.all(writes == 1)
    np.testing.assert_allclose(A, ref, rtol=0, atol=1e-12)
