"""Host check of the in-place streaming addressing (Sec. 4.3) read for the
AA pattern and the esoteric family (Esoteric Twist, Pull, Push): emulated
element by element on a small periodic lattice with a random linear
collision, each pattern must touch every storage element exactly once per
step (so the in-place update is race-free), write exactly the elements each
cell read, and leave after every step the same canonical populations as
pull streaming.  The rules restate the addressing the step kernels use:

* AA: even steps read slot i at x and write slot ibar at x; odd steps read
  slot ibar at x - xi_i and write slot i at x + xi_i.
* esoteric: pair (p, pbar), p of odd index, owns (x + a_p, slot p) and
  (x + a_p + xi_p, slot pbar); Twist a_p = max(-xi_p, 0), Pull a_p = 0,
  Push a_p = -xi_p; even steps read slot i and write slot ibar, odd steps
  swap the slot labels.
"""
import numpy as np
import pytest

import oracle as O


def opp(i):
    return 0 if i == 0 else (i + 1 if i % 2 else i - 1)


def esoteric_offsets(xi, kind):
    """r_i (read node offset) and w_i (write node offset) of each direction."""
    def alpha(v):
        if kind == "twist":
            return np.maximum(-v, 0)
        if kind == "pull":
            return np.zeros_like(v)
        return -v  # push
    q = len(xi)
    r = np.zeros((q, 3), dtype=int)
    w = np.zeros((q, 3), dtype=int)
    for i in range(1, q):
        p = i if i % 2 else opp(i)
        a = alpha(xi[p])
        r[i] = a if i == p else a + xi[p]
        w[i] = a + xi[p] if i == p else a
    return r, w


class Grid:
    def __init__(self, dims):
        self.dims = dims
        self.N = dims[0] * dims[1] * dims[2]

    def node(self, c, off):
        nx, ny, nz = self.dims
        x, y, z = c % nx, (c // nx) % ny, c // (nx * ny)
        return (((z + off[2]) % nz) * ny + (y + off[1]) % ny) * nx + (x + off[0]) % nx


def pattern_rules(xi, pattern):
    """(read(i, parity) -> (slot, offset), write(i, parity) -> (slot, offset),
    layout(i, parity) -> (slot, offset)) where layout is where population i
    of cell x is held at a time of the given parity."""
    zero = np.zeros(3, dtype=int)
    if pattern == "aa":
        def read(i, par):
            return (opp(i), -xi[i]) if par else (i, zero)

        def write(i, par):
            return (i, xi[i]) if par else (opp(i), zero)
        return read, write, read
    r, w = esoteric_offsets(xi, pattern)

    def read(i, par):
        return (opp(i) if par else i), r[i]

    def write(i, par):
        return (i if par else opp(i)), w[i]
    return read, write, read


@pytest.mark.parametrize("pattern", ["aa", "twist", "pull", "push"])
@pytest.mark.parametrize("st", [O.D2Q9, O.D3Q19, O.D3Q27], ids=["D2Q9", "D3Q19", "D3Q27"])
def test_in_place_pattern_is_race_free_and_equals_pull(st, pattern):
    xi, w, _ = O.lattice(st)
    xi = np.asarray(xi, dtype=int)
    q = len(w)
    g = Grid((5, 4, 1) if st == O.D2Q9 else (4, 3, 3))
    rng = np.random.default_rng(7 + st)
    A = rng.standard_normal((q, q)) / q  # a linear stand-in for the collision
    f = rng.standard_normal((q, g.N))
    read, write, layout = pattern_rules(xi, pattern)
    buf = np.full((q, g.N), np.nan)
    for c in range(g.N):
        for i in range(q):
            s, off = layout(i, 0)
            buf[s, g.node(c, off)] = f[i, c]
    assert not np.isnan(buf).any()  # the layout fills every element once
    ref = f.copy()
    for n in range(5):
        par = n % 2
        touched = np.zeros((q, g.N), dtype=int)
        post = {}
        for c in range(g.N):
            rd = [(read(i, par)[0], g.node(c, read(i, par)[1])) for i in range(q)]
            wr = [(write(i, par)[0], g.node(c, write(i, par)[1])) for i in range(q)]
            assert sorted(rd) == sorted(wr)
            for s, e in rd:
                touched[s, e] += 1
            post[c] = A @ np.array([buf[s, e] for s, e in rd])
        assert (touched == 1).all()
        for c, fs in post.items():
            for i in range(q):
                s, off = write(i, par)
                buf[s, g.node(c, off)] = fs[i]
        nxt = np.empty_like(ref)
        for c in range(g.N):
            fs = A @ ref[:, c]
            for i in range(q):
                nxt[i, g.node(c, xi[i])] = fs[i]
        ref = nxt
        got = np.empty_like(ref)
        for c in range(g.N):
            for i in range(q):
                s, off = layout(i, (n + 1) % 2)
                got[i, c] = buf[s, g.node(c, off)]
        assert np.array_equal(got, ref), n


def test_twist_touches_only_the_cell_and_its_positive_neighbours():
    xi, _, _ = O.lattice(O.D3Q27)
    r, w = esoteric_offsets(np.asarray(xi, dtype=int), "twist")
    assert r.min() == 0 and w.min() == 0 and r.max() == 1 and w.max() == 1
    assert np.array_equal(r, np.maximum(-np.asarray(xi), 0))
    assert np.array_equal(w, np.maximum(np.asarray(xi), 0))
