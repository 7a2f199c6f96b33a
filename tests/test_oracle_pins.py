"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

* dense LU brute force (numpy.linalg.solve / matmul) on tiny lines, for the Thomas,
  periodic (Sherman-Morrison) Thomas and transposed solves;
* the closed-form modified wavenumbers of the periodic schemes on Fourier modes;
* Taylor exactness of every scheme row on monomials (which fixes the interior
  coefficients uniquely and the order of each closure), and exactness of the whole
  closed line on low-degree polynomials;
* sixth-order convergence on a smooth periodic function (Sec. 4.2, order-of-accuracy
  study);
* adjoint identities: <D f, g> = <f, D^T g>, and D1^T = -D1, D2^T = D2 on periodic lines;
* the coefficients printed in Eq. cfds and a hand-enumerated layout example
  (``tests/golden``).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def dense(o, n, order, bc, h):
    """Dense A and B assembled from the oracle's bands (wrap-around on cyclic lines)."""
    a, b, c, B7 = o.bands(n, order, bc, h)
    A = np.zeros((n, n)); B = np.zeros((n, n))
    per = bc == "periodic"
    for i in range(n):
        A[i, i] = b[i]
        if i > 0: A[i, i - 1] = a[i]
        elif per: A[i, n - 1] += a[i]
        if i < n - 1: A[i, i + 1] = c[i]
        elif per: A[i, 0] += c[i]
        for t in range(7):
            j = i + t - 3
            if B7[i, t] == 0.0: continue
            if per: j %= n
            assert 0 <= j < n
            B[i, j] += B7[i, t]
    return A, B


# ----------------------------------------------------------------- golden coefficients

def test_first_derivative_coefficients_match_paper(oracle_mod):
    vals = {}
    with open(os.path.join(GOLDEN, "compact_first_derivative.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                name, num, den = line.split()
                vals[name] = int(num) / int(den)
    n, h = 32, 0.1
    a, b, c, B7 = oracle_mod.bands(n, 1, "periodic", h)
    for i in range(n):
        assert a[i] == pytest.approx(vals["alpha"], rel=1e-15)
        assert c[i] == pytest.approx(vals["alpha"], rel=1e-15)
        assert b[i] == 1.0
        np.testing.assert_allclose(
            B7[i], [0, -vals["b"] / (4 * h), -vals["a"] / (2 * h), 0,
                    vals["a"] / (2 * h), vals["b"] / (4 * h), 0], rtol=1e-15)


# ------------------------------------------------------------------ dense brute force

@pytest.mark.parametrize("n", [8, 12, 16, 32])
@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("bc", ["periodic", "closed"])
def test_deriv_matches_dense_lu(oracle_mod, n, order, bc):
    rng = np.random.default_rng(100 + n + 7 * order)
    h = oracle_mod.grid_spacing(n, bc)
    A, B = dense(oracle_mod, n, order, bc, h)
    f = rng.uniform(-1, 1, size=(5, n))
    ref = np.linalg.solve(A, B @ f.T).T
    got = oracle_mod.deriv_lines(f, order, bc, h)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    # the right-hand side alone
    np.testing.assert_allclose(oracle_mod.rhs_lines(f, order, bc, h), (B @ f.T).T,
                               rtol=0, atol=1e-14 * np.max(np.abs(B @ f.T)))


@pytest.mark.parametrize("n", [8, 12, 16, 32])
@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("bc", ["periodic", "closed"])
def test_adjoint_matches_dense_lu(oracle_mod, n, order, bc):
    rng = np.random.default_rng(200 + n + 7 * order)
    h = oracle_mod.grid_spacing(n, bc)
    A, B = dense(oracle_mod, n, order, bc, h)
    g = rng.normal(size=(5, n))
    ref = (B.T @ np.linalg.solve(A.T, g.T)).T
    got = oracle_mod.deriv_adjoint_lines(g, order, bc, h)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("n", [3, 4, 7, 50])
def test_tridiagonal_solver_random_dominant(oracle_mod, periodic, n):
    rng = np.random.default_rng(n + 10 * periodic)
    a = rng.uniform(-1, 1, n); c = rng.uniform(-1, 1, n)
    b = 2.5 + rng.uniform(0, 1, n)
    d = rng.normal(size=n)
    M = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
    if periodic:
        M[0, n - 1] += a[0]; M[n - 1, 0] += c[n - 1]
    ref = np.linalg.solve(M, d)
    got = oracle_mod.tridiag_solve(a, b, c, d, periodic)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.max(np.abs(ref)))


# ------------------------------------------------------- closed form: modified wavenumber

def mod_wavenumber(order, k, h):
    """Fourier symbol of the periodic interior scheme (derived from the stencil)."""
    if order == 1:
        al, a, b = 1 / 3, 14 / 9, 1 / 9
        return (a * np.sin(k * h) + 0.5 * b * np.sin(2 * k * h)) / (h * (1 + 2 * al * np.cos(k * h)))
    al, a, b = 2 / 11, 12 / 11, 3 / 11
    return ((2 * a * (1 - np.cos(k * h)) + 0.5 * b * (1 - np.cos(2 * k * h)))
            / (h * h * (1 + 2 * al * np.cos(k * h))))


@pytest.mark.parametrize("n", [16, 64, 256])
@pytest.mark.parametrize("order", [1, 2])
def test_modified_wavenumber_closed_form(oracle_mod, n, order):
    h = 2 * np.pi / n
    x = np.arange(n) * h
    rng = np.random.default_rng(n + order)
    for k in [1, 2, 3, n // 4, n // 2 - 1]:
        phi = rng.uniform(0, 2 * np.pi)
        f = np.cos(k * x + phi)
        got = oracle_mod.deriv_lines(f[None, :], order, "periodic", h)[0]
        kk = mod_wavenumber(order, k, h)
        ref = -kk * np.sin(k * x + phi) if order == 1 else -kk * np.cos(k * x + phi)
        # rounding scales with the operator norm (the largest symbol over all modes),
        # not with the (possibly small) symbol of this one mode
        kmax = np.max(np.abs(mod_wavenumber(order, np.arange(n // 2 + 1), h)))
        assert np.max(np.abs(got - ref)) <= 1e-13 * kmax


def test_modified_wavenumber_multidirection_field(oracle_mod):
    """A mode cos(kx x + ky y + kz z + phi) differentiated along each direction."""
    nz, ny, nx = 16, 32, 64
    kx, ky, kz, phi = 5, 3, 2, 0.7
    X = np.arange(nx) * 2 * np.pi / nx
    Y = np.arange(ny) * 2 * np.pi / ny
    Z = np.arange(nz) * 2 * np.pi / nz
    arg = kx * X[None, None, :] + ky * Y[None, :, None] + kz * Z[:, None, None] + phi
    f = np.cos(arg)
    for d, k, n in (("x", kx, nx), ("y", ky, ny), ("z", kz, nz)):
        got = oracle_mod.deriv(f, d, 1, "periodic")
        ref = -mod_wavenumber(1, k, 2 * np.pi / n) * np.sin(arg)
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
        got2 = oracle_mod.deriv(f, d, 2, "periodic")
        ref2 = -mod_wavenumber(2, k, 2 * np.pi / n) * np.cos(arg)
        assert np.max(np.abs(got2 - ref2)) <= 1e-12 * np.max(np.abs(ref2))


# ----------------------------------------------------------- Taylor / polynomial exactness

def _row_residual(o, n, order, bc, h, i, p, x0):
    """Residual of row i of A u' = B f for f = (x - x0)^p, in exact rational arithmetic
    on the coefficients returned by the oracle."""
    a, b, c, B7 = o.bands(n, order, bc, h)
    def f(j): return Fraction(j * 1) ** p if p > 0 else Fraction(1)
    # derivative of x^p at grid index j (x_j = j*h, x0 = 0): order 1 or 2
    def df(j):
        if order == 1:
            return Fraction(p) * Fraction(j) ** (p - 1) if p >= 1 else Fraction(0)
        return Fraction(p * (p - 1)) * Fraction(j) ** (p - 2) if p >= 2 else Fraction(0)
    # work in units h = 1 with exact rationals: scale B by h^order
    hs = Fraction(h) ** order
    lhs = Fraction(b[i]) * df(i - x0)
    if i > 0: lhs += Fraction(a[i]) * df(i - 1 - x0)
    if i < n - 1: lhs += Fraction(c[i]) * df(i + 1 - x0)
    rhs = Fraction(0)
    for t in range(7):
        j = i + t - 3
        if B7[i, t] != 0.0:
            rhs += Fraction(B7[i, t]) * hs * f(j - x0)
    return float(lhs - rhs), float(abs(lhs) + 1)


# (row, exact-through degree) for each scheme's rows; the interior row is exact through
# degree 6 (first derivative) and 7 (second derivative): that alone fixes alpha, a, b.
ROWS = {1: [(0, 3), (1, 4), ("mid", 6), (-2, 4), (-1, 3)],
        2: [(0, 4), (1, 5), ("mid", 7), (-2, 5), (-1, 4)]}


@pytest.mark.parametrize("order", [1, 2])
def test_rows_taylor_exact_to_stated_degree(oracle_mod, order):
    n = 16
    h = 1.0  # power of two: the coefficients are then exact rationals of the scheme
    for row, deg in ROWS[order]:
        i = n // 2 if row == "mid" else (row % n)
        x0 = i  # expand around the row's own node
        for p in range(0, deg + 1):
            r, s = _row_residual(oracle_mod, n, order, "closed", h, i, p, x0)
            assert abs(r) <= 1e-12 * s, (order, row, p, r)
        # and not exact one degree higher (pins the stated order of each closure);
        # odd/even symmetry makes the centred rows exact one more degree
        p = deg + 1
        r, s = _row_residual(oracle_mod, n, order, "closed", h, i, p, x0)
        if row in (0, -1):
            assert abs(r) > 1e-6, (order, row, p)
        else:
            r2, s2 = _row_residual(oracle_mod, n, order, "closed", h, i, p + 1, x0)
            assert abs(r) > 1e-6 or abs(r2) > 1e-6, (order, row, p)


@pytest.mark.parametrize("order,maxdeg", [(1, 3), (2, 4)])
def test_closed_line_exact_on_polynomials(oracle_mod, order, maxdeg):
    n = 40
    h = 2.0 / (n - 1)
    x = -1.0 + np.arange(n) * h
    for p in range(0, maxdeg + 1):
        f = x ** p
        if order == 1:
            ref = p * x ** (p - 1) if p else np.zeros(n)
        else:
            ref = p * (p - 1) * x ** (p - 2) if p >= 2 else np.zeros(n)
        got = oracle_mod.deriv_lines(f[None, :], order, "closed", h)[0]
        # rounding scale: largest absolute row sum of B times max|f|
        _, _, _, B7 = oracle_mod.bands(n, order, "closed", h)
        scale = np.max(np.sum(np.abs(B7), axis=1)) * max(1.0, np.max(np.abs(f)))
        assert np.max(np.abs(got - ref)) <= 1e-13 * scale, p
    # one degree higher is no longer exact at the boundary
    f = x ** (maxdeg + 1)
    got = oracle_mod.deriv_lines(f[None, :], order, "closed", h)[0]
    ref = ((maxdeg + 1) * x ** maxdeg if order == 1
           else (maxdeg + 1) * maxdeg * x ** (maxdeg - 1))
    assert np.max(np.abs(got - ref)) > 1e-6


def test_sixth_order_convergence_periodic(oracle_mod):
    """Error against the analytic derivative falls as h^6 (order-of-accuracy study of
    Sec. 4.2 for n = 32..256)."""
    for order in (1, 2):
        errs = []
        ns = [32, 64, 128]
        for n in ns:
            h = 2 * np.pi / n
            x = np.arange(n) * h
            f = np.sin(x) + 0.5 * np.cos(2 * x + 0.3)
            ex = (np.cos(x) - np.sin(2 * x + 0.3)) if order == 1 else \
                 (-np.sin(x) - 2.0 * np.cos(2 * x + 0.3))
            got = oracle_mod.deriv_lines(f[None, :], order, "periodic", h)[0]
            errs.append(np.max(np.abs(got - ex)))
        rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
        for r in rates:
            assert 5.7 < r < 6.3, (order, errs, rates)


# ------------------------------------------------------------------- adjoint identities

@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("bc", ["periodic", "closed"])
@pytest.mark.parametrize("n", [16, 64, 257])
def test_adjoint_dot_product(oracle_mod, order, bc, n):
    rng = np.random.default_rng(n * order)
    h = oracle_mod.grid_spacing(n, bc)
    f = rng.uniform(-1, 1, (3, n)); g = rng.normal(size=(3, n))
    Df = oracle_mod.deriv_lines(f, order, bc, h)
    DTg = oracle_mod.deriv_adjoint_lines(g, order, bc, h)
    lhs = np.sum(Df * g, axis=1); rhs = np.sum(f * DTg, axis=1)
    scale = np.sum(np.abs(Df * g), axis=1)
    assert np.all(np.abs(lhs - rhs) <= 1e-13 * scale)


@pytest.mark.parametrize("n", [16, 96])
def test_periodic_adjoint_symmetry(oracle_mod, n):
    rng = np.random.default_rng(n)
    h = 2 * np.pi / n
    g = rng.normal(size=(4, n))
    d1 = oracle_mod.deriv_lines(g, 1, "periodic", h)
    d1t = oracle_mod.deriv_adjoint_lines(g, 1, "periodic", h)
    np.testing.assert_allclose(d1t, -d1, rtol=0, atol=1e-13 * np.max(np.abs(d1)))
    d2 = oracle_mod.deriv_lines(g, 2, "periodic", h)
    d2t = oracle_mod.deriv_adjoint_lines(g, 2, "periodic", h)
    np.testing.assert_allclose(d2t, d2, rtol=0, atol=1e-13 * np.max(np.abs(d2)))


# ----------------------------------------------------------------------------- layouts

def test_layout_hand_enumerated_example(oracle_mod):
    shape = (2, 2, 3)  # (nz, ny, nx)
    cart = np.arange(12, dtype=np.float64).reshape(shape)  # v = x + 3y + 6z
    want = {}
    with open(os.path.join(GOLDEN, "layout_tiny.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                parts = line.split()
                want[parts[0]] = [float(v) for v in parts[1:]]
    for d in "xyz":
        lay = oracle_mod.to_layout(cart, d, 2)
        assert lay.tolist() == want[d], d
        back = oracle_mod.from_layout(lay, d, shape, 2)
        assert np.array_equal(back, cart)


def test_layout_round_trip_and_derivative_consistency(oracle_mod):
    rng = np.random.default_rng(3)
    shape = (8, 16, 32)
    cart = rng.uniform(-1, 1, shape)
    for d in "xyz":
        lay = oracle_mod.to_layout(cart, d, 8)
        assert np.array_equal(oracle_mod.from_layout(lay, d, shape, 8), cart)
    # derivative along y via lines equals the same derivative along x of the transposed field
    dy = oracle_mod.deriv(cart, "y", 1, "periodic")
    dx_t = oracle_mod.deriv(np.ascontiguousarray(cart.transpose(0, 2, 1)), "x", 1, "periodic")
    assert np.array_equal(dy, dx_t.transpose(0, 2, 1))


# --------------------------------------------------- transport equation (Sec. 5, Eq. mom-comps)

def _modes_eval(modes, grids):
    X, Y, Z = grids
    out = np.zeros(np.broadcast(X, Y, Z).shape)
    for amp, (kx, ky, kz), ph in modes:
        out = out + amp * np.cos(kx * X + ky * Y + kz * Z + ph)
    return out


def _modes_product(ma, mb):
    """cos(a) cos(b) = (cos(a + b) + cos(a - b)) / 2, term by term."""
    out = []
    for a1, k1, p1 in ma:
        for a2, k2, p2 in mb:
            out.append((0.5 * a1 * a2, tuple(u + v for u, v in zip(k1, k2)), p1 + p2))
            out.append((0.5 * a1 * a2, tuple(u - v for u, v in zip(k1, k2)), p1 - p2))
    return out


def _modes_deriv(modes, axis, order, hs):
    """The periodic compact derivative of a sum of grid modes, from the Fourier symbol alone:
    D1 cos(t) = -K1 sin(t) = K1 cos(t + pi/2), D2 cos(t) = -K2 cos(t) (any integer wavenumber
    is an eigenvector of the circulant scheme)."""
    out = []
    for amp, k, ph in modes:
        kk = mod_wavenumber(order, k[axis], hs[axis])
        out.append((amp * kk, k, ph + np.pi / 2) if order == 1 else (-amp * kk, k, ph))
    return out


def test_transport_rhs_closed_form_fourier(oracle_mod):
    """Every term of Eq. mom-comps on fields made of a constant plus one 3D Fourier mode each:
    the expected values use only the closed-form symbols (products expanded into modes)."""
    nz, ny, nx = 12, 16, 20
    hs = (2 * np.pi / nx, 2 * np.pi / ny, 2 * np.pi / nz)
    grids = (np.arange(nx)[None, None, :] * hs[0], np.arange(ny)[None, :, None] * hs[1],
             np.arange(nz)[:, None, None] * hs[2])
    spec = [(0.7, 1.3, (2, 1, 3), 0.4), (-0.4, 0.9, (1, 3, 2), 1.1), (0.25, 1.1, (3, 2, 1), -0.6)]
    modes = [[(c, (0, 0, 0), 0.0), (a, k, p)] for c, a, k, p in spec]
    u = [_modes_eval(m, grids) for m in modes]
    nu = 0.03
    got = oracle_mod.transport_rhs(u, nu, "periodic")
    for i in range(3):
        ref = np.zeros((nz, ny, nx))
        scale = 0.0
        for j in range(3):
            conv = u[j] * _modes_eval(_modes_deriv(modes[i], j, 1, hs), grids)
            cons = _modes_eval(_modes_deriv(_modes_product(modes[j], modes[i]), j, 1, hs), grids)
            visc = _modes_eval(_modes_deriv(modes[i], j, 2, hs), grids)
            ref += -0.5 * (conv + cons) + nu * visc
            scale = max(scale, np.max(np.abs(conv)), np.max(np.abs(cons)), nu * np.max(np.abs(visc)))
            term = oracle_mod.transport_term(u[i], u[j], "xyz"[j], nu, "periodic")
            np.testing.assert_allclose(term, -0.5 * (conv + cons) + nu * visc, rtol=0, atol=1e-12 * scale)
        np.testing.assert_allclose(got[i], ref, rtol=0, atol=1e-12 * scale)


@pytest.mark.parametrize("j", ["x", "y", "z"])
def test_transport_skew_symmetric_energy_identity(oracle_mod, j):
    """On periodic lines D1 is skew (A symmetric, B antisymmetric, both circulant), so the
    convective part of each term group conserves energy for ANY fields:
    <u_i, u_j D1 u_i> + <u_i, D1 (u_j u_i)> = <u_i u_j, D1 u_i> - <D1 u_i, u_j u_i> = 0,
    and the viscous part is dissipative (<u_i, D2 u_i> < 0 for a non-constant u_i)."""
    rng = np.random.default_rng(11)
    shape = (10, 14, 18)
    ui, uj = rng.uniform(-1, 1, shape), rng.uniform(-1, 1, shape)
    t0 = oracle_mod.transport_term(ui, uj, j, 0.0, "periodic")
    conv = uj * oracle_mod.deriv(ui, j, 1, "periodic")
    bound = 1e-13 * np.sum(np.abs(ui) * (np.abs(conv) + np.abs(t0))) + 1e-300
    assert abs(np.sum(ui * t0)) <= bound
    # the same for i = j
    tj = oracle_mod.transport_term(uj, uj, j, 0.0, "periodic")
    assert abs(np.sum(uj * tj)) <= 1e-13 * np.sum(np.abs(uj) * (np.abs(uj) * 10 + np.abs(tj)))
    # the identity is not trivial: the convective half alone carries energy
    assert abs(np.sum(ui * conv)) > 1e3 * bound
    t1 = oracle_mod.transport_term(ui, uj, j, 0.5, "periodic")
    assert np.sum(ui * t1) < -1e3 * bound


# ------------------------------------- compact filter and mid-point interpolation (Lele 1992)
# The coefficients are pinned by their defining conditions, evaluated on the oracle's own band
# rows in exact rational arithmetic: a filter row keeps polynomials up to its order and removes
# the grid's odd-even mode; the interpolation row is exact at the mid-point through degree 5.
# The solved operators are pinned against their Fourier symbols (from the same rows) and against
# dense LU.

AF = 0.375   # a dyadic filter parameter: the coefficients are then exact binary fractions


def _filter_row_residual(o, n, bc, i, p, x0):
    """Row i of the filter, alpha g[i-1] + g[i] + alpha g[i+1] = sum B7 f, on f = g = (x - x0)^p."""
    a, b, c, B7 = o.bands(n, o.FILTER, bc, AF)
    def f(j): return Fraction(j) ** p if p > 0 else Fraction(1)
    lhs = Fraction(b[i]) * f(i - x0)
    if i > 0 or bc == "periodic": lhs += Fraction(a[i]) * f(i - 1 - x0)
    if i < n - 1 or bc == "periodic": lhs += Fraction(c[i]) * f(i + 1 - x0)
    rhs = sum(Fraction(B7[i, t]) * f(i + t - 3 - x0) for t in range(7) if B7[i, t] != 0.0)
    return lhs - rhs


@pytest.mark.parametrize("row,deg", [("mid", 3), (1, 1), (-2, 1), (0, 99), (-1, 99)])
def test_filter_rows_keep_polynomials_to_their_order(oracle_mod, row, deg):
    n = 16
    i = n // 2 if row == "mid" else row % n
    for p in range(0, min(deg, 6) + 1):
        assert _filter_row_residual(oracle_mod, n, "closed", i, p, i) == 0, (row, p)
    if deg < 99:   # exactly that order: the next even degree is not kept
        assert _filter_row_residual(oracle_mod, n, "closed", i, deg + 1, i) != 0
    a, b, c, B7 = oracle_mod.bands(n, oracle_mod.FILTER, "closed", AF)
    if row in (0, -1):   # the end values are kept: g = f with no coupling
        assert a[i] == 0 and c[i] == 0 and b[i] == 1 and B7[i, 3] == 1 and np.count_nonzero(B7[i]) == 1
    else:                # the right-hand side of the row removes the odd-even mode
        assert sum(Fraction(B7[i, t]) * (-1) ** t for t in range(7)) == 0
        assert a[i] == AF and c[i] == AF


def _symbol(o, op, n, bc, param, k, shift=0.0):
    """Fourier symbol of the uniform row of an operator from the oracle's band: the factor that
    maps cos(k x_j + phi) to cos(k (x_j + shift h) + phi) (real for symmetric rows)."""
    a, b, c, B7 = o.bands(n, op, bc, param)
    i = n // 2
    th = 2 * np.pi * k / n
    num = sum(B7[i, t] * np.exp(1j * th * (t - 3 - shift)) for t in range(7))
    den = a[i] * np.exp(-1j * th) + b[i] + c[i] * np.exp(1j * th)
    return num / den


@pytest.mark.parametrize("n", [16, 64])
def test_filter_transfer_function_on_fourier_modes(oracle_mod, n):
    x = np.arange(n) * 2 * np.pi / n
    for k in [0, 1, 3, n // 4, n // 2 - 1, n // 2]:
        phi = 0.3 * k + 0.1
        f = np.cos(k * x + phi)
        T = _symbol(oracle_mod, oracle_mod.FILTER, n, "periodic", AF, k)
        assert abs(T.imag) <= 1e-15
        got = oracle_mod.filter_lines(f[None, :], AF, "periodic")[0]
        np.testing.assert_allclose(got, T.real * f, rtol=0, atol=1e-13)
        if k == 0:
            assert abs(T.real - 1.0) <= 1e-15
        if k == n // 2:   # the odd-even mode is removed
            assert np.max(np.abs(got)) <= 1e-14


@pytest.mark.parametrize("n", [16, 33])
@pytest.mark.parametrize("bc", ["periodic", "closed"])
def test_filter_matches_dense_lu_and_adjoint(oracle_mod, n, bc):
    rng = np.random.default_rng(n + 3 * (bc == "closed"))
    A, B = dense(oracle_mod, n, oracle_mod.FILTER, bc, AF)
    f = rng.uniform(-1, 1, (4, n))
    ref = np.linalg.solve(A, B @ f.T).T
    np.testing.assert_allclose(oracle_mod.filter_lines(f, AF, bc), ref, rtol=0, atol=1e-14)
    refT = (B.T @ np.linalg.solve(A.T, f.T)).T
    np.testing.assert_allclose(oracle_mod.filter_adjoint_lines(f, AF, bc), refT, rtol=0, atol=1e-14)
    if bc == "periodic":   # A and B symmetric circulant: the filter is its own transpose
        np.testing.assert_allclose(refT, ref, rtol=0, atol=1e-14)


def test_interp_row_exact_at_the_midpoint_through_degree_5(oracle_mod):
    n = 16
    a, b, c, B7 = oracle_mod.bands(n, oracle_mod.INTERP, "periodic", 1.0)
    i = n // 2
    half = Fraction(1, 2)

    def residual(p):
        def f(x): return x ** p if p > 0 else Fraction(1)
        # g[j] sits at x_j + 1/2 (units of h, around x_i = 0)
        lhs = Fraction(a[i]) * f(-1 + half) + Fraction(b[i]) * f(half) + Fraction(c[i]) * f(1 + half)
        rhs = sum(Fraction(B7[i, t]) * f(Fraction(t - 3)) for t in range(7) if B7[i, t] != 0.0)
        return lhs - rhs
    # alpha = 3/10 and b/2 = 1/20 are not binary fractions: exact up to their rounding
    for p in range(6):
        assert abs(float(residual(p))) <= 1e-15 * 2.5 ** p, p
    assert abs(float(residual(6))) > 1e-3


@pytest.mark.parametrize("n", [16, 48])
def test_interp_transfer_function_and_dense_lu(oracle_mod, n):
    x = np.arange(n) * 2 * np.pi / n
    h = 2 * np.pi / n
    for k in [0, 1, 2, n // 4, n // 2 - 1]:
        phi = 0.7 - 0.2 * k
        T = _symbol(oracle_mod, oracle_mod.INTERP, n, "periodic", 1.0, k, shift=0.5)
        assert abs(T.imag) <= 1e-15
        got = oracle_mod.interp_lines(np.cos(k * x + phi)[None, :])[0]
        np.testing.assert_allclose(got, T.real * np.cos(k * (x + h / 2) + phi), rtol=0, atol=1e-13)
        # the transpose takes mid-point data back to the nodes with the same factor
        back = oracle_mod.interp_adjoint_lines(np.cos(k * (x + h / 2) + phi)[None, :])[0]
        np.testing.assert_allclose(back, T.real * np.cos(k * x + phi), rtol=0, atol=1e-13)
    rng = np.random.default_rng(n)
    A, B = dense(oracle_mod, n, oracle_mod.INTERP, "periodic", 1.0)
    f = rng.uniform(-1, 1, (3, n))
    np.testing.assert_allclose(oracle_mod.interp_lines(f), np.linalg.solve(A, B @ f.T).T, rtol=0, atol=1e-14)
    np.testing.assert_allclose(oracle_mod.interp_adjoint_lines(f), (B.T @ np.linalg.solve(A.T, f.T)).T,
                               rtol=0, atol=1e-14)


def test_interp_sixth_order_and_filter_parameter_refused(oracle_mod):
    errs = []
    for n in (32, 64, 128):
        h = 2 * np.pi / n
        x = np.arange(n) * h
        f = np.sin(x) + 0.5 * np.cos(2 * x + 0.3)
        ex = np.sin(x + h / 2) + 0.5 * np.cos(2 * (x + h / 2) + 0.3)
        errs.append(np.max(np.abs(oracle_mod.interp_lines(f[None, :])[0] - ex)))
    for e0, e1 in zip(errs, errs[1:]):
        assert 5.7 < math.log2(e0 / e1) < 6.3, errs
    with pytest.raises(ValueError):
        oracle_mod.bands(16, oracle_mod.FILTER, "periodic", 0.5)


# Closed lines: n nodes give n - 1 mid-points.  The closure rows (the first mid-point and its
# mirror) are pinned by their defining conditions -- exact at their mid-point for polynomials
# through degree 4 and not degree 5 -- on the oracle's own band rows in rational arithmetic;
# the last row is a zero row; the solved operator is pinned by dense LU and by its order of
# convergence on a smooth non-periodic function.
@pytest.mark.parametrize("row", [0, -2, 1, -3])
def test_interp_closed_rows_exact_to_their_degree(oracle_mod, row):
    n = 16
    a, b, c, B7 = oracle_mod.bands(n, oracle_mod.INTERP, "closed", 1.0)
    i = row % n
    half = Fraction(1, 2)

    def residual(p):
        def f(x): return x ** p if p > 0 else Fraction(1)
        x0 = Fraction(i)   # g[j] sits at x_j + 1/2, f[j] at x_j (units of h)
        lhs = Fraction(b[i]) * f(x0 + half)
        if i > 0: lhs += Fraction(a[i]) * f(x0 - 1 + half)
        if i < n - 1: lhs += Fraction(c[i]) * f(x0 + 1 + half)
        rhs = sum(Fraction(B7[i, t]) * f(x0 + t - 3) for t in range(7) if B7[i, t] != 0.0)
        return lhs - rhs
    deg = 4 if row in (0, -2) else 5    # closures through degree 4, interior rows through 5
    for p in range(deg + 1):
        assert abs(float(residual(p))) <= 1e-15 * 16.0 ** p, (row, p)
    assert abs(float(residual(deg + 1))) > 1e-3, row


def test_interp_closed_zero_row_dense_lu_and_fifth_order(oracle_mod):
    for n in (16, 33):
        a, b, c, B7 = oracle_mod.bands(n, oracle_mod.INTERP, "closed", 1.0)
        assert a[n - 1] == 0 and c[n - 1] == 0 and c[n - 2] == 0 and b[n - 1] == 1
        assert not np.any(B7[n - 1])
        rng = np.random.default_rng(n)
        A, B = dense(oracle_mod, n, oracle_mod.INTERP, "closed", 1.0)
        f = rng.uniform(-1, 1, (3, n))
        got = oracle_mod.interp_lines(f, "closed")
        np.testing.assert_allclose(got, np.linalg.solve(A, B @ f.T).T, rtol=0, atol=1e-14)
        assert not np.any(got[:, -1])
        back = oracle_mod.interp_adjoint_lines(f, "closed")
        np.testing.assert_allclose(back, (B.T @ np.linalg.solve(A.T, f.T)).T, rtol=0, atol=1e-14)
        f2 = f.copy()
        f2[:, -1] = 7.0   # the last slot is no mid-point: the transpose does not read it
        np.testing.assert_array_equal(oracle_mod.interp_adjoint_lines(f2, "closed"), back)
    # order of convergence: the closures (exact through degree 4) make it five near the ends
    errs = []
    for n in (33, 65, 129, 257):
        x = np.linspace(0.0, 2 * np.pi, n)
        h = x[1] - x[0]
        f = np.sin(x) + 0.5 * np.cos(2 * x + 0.3)
        xm = x[:-1] + h / 2
        ex = np.sin(xm) + 0.5 * np.cos(2 * xm + 0.3)
        errs.append(np.max(np.abs(oracle_mod.interp_lines(f[None, :], "closed")[0, :-1] - ex)))
    for e0, e1 in zip(errs, errs[1:]):
        assert 4.8 < math.log2(e0 / e1) < 5.8, errs
