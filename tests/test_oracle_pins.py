"""Pins of the CPU oracle to facts outside itself (closed forms, invariants,
brute force, published values).  CPU only."""
import os

import numpy as np
import pytest
from numpy.polynomial import polynomial as P

import dns_synth
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ------------------------------------------------------------------ grid

@pytest.mark.parametrize("My", [9, 17, 33, 65])
def test_nodes_are_flipped_gauss_lobatto(My):
    y, _, _, _ = oracle.grid(My)
    j = np.arange(My)
    assert np.allclose(y, np.cos(np.pi * (My - 1 - j) / (My - 1)), atol=1e-15, rtol=0)
    assert y[0] == -1.0 and y[-1] == 1.0 and np.all(np.diff(y) > 0)


@pytest.mark.parametrize("My", [9, 17, 33, 65])
def test_derivatives_exact_on_polynomials(My):
    y, D1, D2, _ = oracle.grid(My)
    for p in range(My):
        c = np.zeros(p + 1); c[p] = 1.0
        f = P.polyval(y, c)
        d1 = P.polyval(y, P.polyder(c, 1))
        d2 = P.polyval(y, P.polyder(c, 2))
        tol1 = 1e-14 * My ** 2 * max(1.0, np.abs(d1).max())
        tol2 = 1e-14 * My ** 4 * max(1.0, np.abs(d2).max())
        assert np.abs(D1 @ f - d1).max() < tol1, p
        assert np.abs(D2 @ f - d2).max() < tol2, p


@pytest.mark.parametrize("My", [9, 17, 33, 49])
def test_clamped_d4_exact_on_clamped_polynomials(My):
    """D4c is exact on (1-y^2)^2 y^p for p <= My-3 (Weideman & Reddy clamped
    fourth derivative cited in Sec. 2)."""
    _, _, _, D4c = oracle.grid(My)
    # nodes in extended precision, so the test data sit on the exact nodes
    j = np.arange(1, My - 1, dtype=np.longdouble)
    yi = -np.cos(np.pi * j / np.longdouble(My - 1))
    D4l = D4c.astype(np.longdouble)
    wpoly = np.array([1.0, 0.0, -2.0, 0.0, 1.0], dtype=np.longdouble)  # (1 - y^2)^2
    for p in range(My - 2):
        c = np.zeros(p + 1, dtype=np.longdouble); c[p] = 1.0
        full = P.polymul(wpoly, c)
        exact = P.polyval(yi, P.polyder(full, 4))
        vals = ((1 - yi) * (1 + yi)) ** 2 * yi ** p   # factored: no cancellation at the walls
        got = D4l @ vals          # extended-precision matvec: only D4c's own rounding remains
        bound = 4 * np.finfo(float).eps * (np.abs(D4l) @ np.abs(vals)) + 1e-14 * np.abs(exact).max()
        assert np.all(np.abs(got - exact) < bound), p


@pytest.mark.parametrize("My", [9, 17, 33, 65])
def test_clenshaw_curtis_exact(My):
    y, _, _, _ = oracle.grid(My)
    w = oracle.cc_weights(My)
    for p in range(My):
        exact = (1 - (-1) ** (p + 1)) / (p + 1)
        assert abs(w @ y ** p - exact) < 1e-14


def test_truncation_matches_paper_mode_counts():
    """Dealiased mode counts of Table geometry3: 2K+1 = Nx with K = (M-1)//3."""
    for mx, my, nx, ny in _read_golden("geometry3_modes.txt"):
        K = dns_synth.truncation(int(mx))
        assert 2 * K + 1 == int(nx)
        assert int(my) - 2 == int(ny)


# ------------------------------------------------------------- operators

@pytest.mark.parametrize("My,k2,dt,re,h", [(17, 2.5, 0.01, 400.0, 0.5),
                                          (33, 7.3, 0.01, 400.0, 1.0),
                                          (33, 0.0, 0.005, 1650.0, 1.0)])
def test_eta_operator_closed_form(My, k2, dt, re, h):
    """(I - g Delta) P_eta = -h dt I on polynomials vanishing at the walls, and
    M_eta = 2 (I - g Delta)^{-1} - I = -I - (2 / (h dt)) P_eta (Eq. CN2)."""
    y, _, _, _ = oracle.grid(My)
    yi = y[1:-1]
    g = h * dt / (2 * re)
    Mv, Pv, Me, Pe = oracle.cn_operators(My, [k2], dt, re, h)
    for p in range(My - 3):
        eta = P.polymul([1.0, 0.0, -1.0], np.eye(p + 1)[p])         # (1 - y^2) y^p
        rhs = P.polyval(yi, eta) - g * (P.polyval(yi, P.polyder(eta, 2)) - k2 * P.polyval(yi, eta))
        got = Pe[0] @ rhs
        assert np.abs(got + h * dt * P.polyval(yi, eta)).max() < 1e-12 * h * dt, p
    assert np.abs(Me[0] + np.eye(My - 2) + (2.0 / (h * dt)) * Pe[0]).max() < 1e-12


@pytest.mark.parametrize("My,k2,dt,re,h", [(17, 2.5, 0.01, 400.0, 0.5),
                                          (33, 7.3, 0.01, 400.0, 1.0),
                                          (41, 1.0, 0.005, 1650.0, 0.5)])
def test_v_operator_closed_form(My, k2, dt, re, h):
    """For clamped polynomials v = (1-y^2)^2 y^p, (Delta - g Delta Delta) v is a
    known polynomial and P_v maps it to -h dt v; and M_v = 2 A^{-1} Delta - I =
    -I - (2/(h dt)) P_v Delta (Eq. CN1 multiplied through by Delta)."""
    y, D1, D2, _ = oracle.grid(My)
    yi = y[1:-1]
    g = h * dt / (2 * re)
    Mv, Pv, Me, Pe = oracle.cn_operators(My, [k2], dt, re, h)
    for p in range(My - 5):
        v = P.polymul([1.0, 0.0, -2.0, 0.0, 1.0], np.eye(p + 1)[p])
        lap = P.polyval(yi, P.polyder(v, 2)) - k2 * P.polyval(yi, v)
        bih = (P.polyval(yi, P.polyder(v, 4)) - 2 * k2 * P.polyval(yi, P.polyder(v, 2))
               + k2 * k2 * P.polyval(yi, v))
        rhs = lap - g * bih
        got = Pv[0] @ rhs
        assert np.abs(got + h * dt * P.polyval(yi, v)).max() < 1e-11 * h * dt, p
    Delta = D2[1:-1, 1:-1] - k2 * np.eye(My - 2)
    R = Mv[0] + np.eye(My - 2) + (2.0 / (h * dt)) * (Pv[0] @ Delta)
    assert np.abs(R).max() < 1e-9


def test_eta_operator_eigenvalues():
    """M_eta has the CN amplification factors (1 + g mu)/(1 - g mu) of the
    eigenvalues mu = lambda - k^2 of the Dirichlet Laplacian."""
    My, k2, dt, re, h = 25, 3.0, 0.01, 300.0, 1.0
    _, _, D2, _ = oracle.grid(My)
    lam = np.linalg.eigvals(D2[1:-1, 1:-1]).real
    g = h * dt / (2 * re)
    mu = lam - k2
    want = np.sort((1 + g * mu) / (1 - g * mu))
    _, _, Me, _ = oracle.cn_operators(My, [k2], dt, re, h)
    got = np.sort(np.linalg.eigvals(Me[0]).real)
    assert np.abs(got - want).max() < 1e-10


# ------------------------------------------------- transforms / products

def _full_spectrum(c, Kx, Kz):
    """Kept half-spectrum c[m+Kz, n] -> dict (n, m) -> coefficient, both signs of n,
    the n = 0 column replaced by its Hermitian part."""
    out = {}
    for mi in range(2 * Kz + 1):
        m = mi - Kz
        for n in range(Kx + 1):
            if n == 0:
                val = 0.5 * (c[mi, 0] + np.conj(c[2 * Kz - mi, 0]))
                out[(0, m)] = val
            else:
                out[(n, m)] = c[mi, n]
                out[(-n, -m)] = np.conj(c[mi, n])
    return out


@pytest.mark.parametrize("mx,mz", [(4, 4), (7, 10), (10, 7), (16, 13)])
def test_dealiased_product_equals_triad_sum(mx, mz):
    """The pseudo-spectral product with 2/3-rule truncation equals the exact
    convolution sum over kept triads (Orszag 1971's 2/3 rule, Sec. 3.2)."""
    ch = oracle.Channel.__new__(oracle.Channel)
    ch.mx, ch.mz = mx, mz
    ch.Kx, ch.Kz = (mx - 1) // 3, (mz - 1) // 3
    Kx, Kz = ch.Kx, ch.Kz
    rng = np.random.default_rng(mx * 100 + mz)
    a = rng.normal(size=(2 * Kz + 1, Kx + 1)) + 1j * rng.normal(size=(2 * Kz + 1, Kx + 1))
    b = rng.normal(size=(2 * Kz + 1, Kx + 1)) + 1j * rng.normal(size=(2 * Kz + 1, Kx + 1))
    got = ch.to_spectral(ch.to_physical(a) * ch.to_physical(b))
    A = _full_spectrum(a, Kx, Kz)
    B = _full_spectrum(b, Kx, Kz)
    want = np.zeros_like(a)
    for (n1, m1), va in A.items():
        for (n2, m2), vb in B.items():
            n, m = n1 + n2, m1 + m2
            if 0 <= n <= Kx and abs(m) <= Kz:
                want[m + Kz, n] += va * vb
    assert np.abs(got - want).max() < 1e-13 * np.abs(want).max()


def test_product_aliases_on_too_small_grid():
    """Sensitivity check of the triad test: with M = 2K+1 < 3K+1 the same
    comparison must fail (aliased triads fold back)."""
    K = 3
    ch = oracle.Channel.__new__(oracle.Channel)
    ch.mx, ch.mz, ch.Kx, ch.Kz = 2 * K + 1, 1, K, 0
    rng = np.random.default_rng(1)
    a = (rng.normal(size=(1, K + 1)) + 1j * rng.normal(size=(1, K + 1)))
    got = ch.to_spectral(ch.to_physical(a) * ch.to_physical(a))
    A = _full_spectrum(a, K, 0)
    want = np.zeros_like(a)
    for (n1, _), va in A.items():
        for (n2, _), vb in A.items():
            if 0 <= n1 + n2 <= K:
                want[0, n1 + n2] += va * vb
    assert np.abs(got - want).max() > 1e-3


# ----------------------------------------------------------- time scheme

def _kutta_rk3(f, x, dt):
    k1 = f(x)
    k2 = f(x + 0.5 * dt * k1)
    k3 = f(x - dt * k1 + 2.0 * dt * k2)
    return x + dt * (k1 + 4.0 * k2 + k3) / 6.0


def test_cn_rk3_without_viscosity_is_kutta():
    """With the viscous operator off, the three CN/RK3 sub-steps of Sec. 3.1
    reduce to Kutta's classical third-order method."""
    f = lambda x: np.sin(x) + x * x
    dt = 0.1
    for x0 in (0.3, -1.1, 2.0):
        got = oracle.cn_rk3(x0, lambda x: -f(x), lambda xt, Ft, h, s: xt - h * dt * Ft)
        assert abs(got - _kutta_rk3(f, x0, dt)) < 1e-15


def test_cn_rk3_third_order_in_dt():
    f = lambda x: -x * x
    exact = lambda t: 1.0 / (1.0 + t)       # x' = -x^2, x(0) = 1
    errs = []
    for nsteps in (10, 20, 40):
        dt = 1.0 / nsteps
        x = 1.0
        for _ in range(nsteps):
            x = oracle.cn_rk3(x, lambda x: -f(x), lambda xt, Ft, h, s: xt - h * dt * Ft)
        errs.append(abs(x - exact(1.0)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 2.8)


# ------------------------------------------------------- whole-step pins

def _state(st):
    return tuple(st[k] for k in ("v", "eta", "U", "W"))


def test_laminar_couette_is_steady():
    ch = oracle.Channel(16, 33, 16, 1.75 * np.pi, 1.2 * np.pi, 400.0, 0.01, "couette")
    x = _state(dns_synth.make_state(16, 33, 16, 1.75 * np.pi, 1.2 * np.pi, "couette", 1, 0, 0.0))
    y = ch.step(x, 10)
    assert np.abs(y[2] - x[2]).max() < 1e-14
    assert np.abs(y[0]).max() == 0.0 and np.abs(y[3]).max() == 0.0
    s = ch.stats(y)
    assert abs(s["tau_bottom"][0] - 1.0) < 1e-13 and abs(s["tau_top"][0] - 1.0) < 1e-13


def test_laminar_poiseuille_is_steady_with_gamma_two_over_re():
    re = 1650.0
    ch = oracle.Channel(16, 33, 16, 2 * np.pi, np.pi, re, 0.005, "poiseuille")
    x = _state(dns_synth.make_state(16, 33, 16, 2 * np.pi, np.pi, "poiseuille", 1, 0, 0.0))
    y = ch.step(x, 10)
    assert np.abs(y[2] - x[2]).max() < 1e-14
    assert abs(ch.last_gamma[0] - 2.0 / re) < 1e-15
    assert abs(ch.stats(y)["bulk_flux"][0] - 4.0 / 3.0) < 1e-14


@pytest.mark.parametrize("u_wall", [0.5, -2.0])
def test_laminar_couette_at_other_wall_speeds_is_steady(u_wall):
    """U = U_w y with walls at +-U_w is a steady solution; its wall shear is U_w."""
    ch = oracle.Channel(16, 25, 16, 1.75 * np.pi, 1.2 * np.pi, 400.0, 0.01, "couette", u_wall=u_wall)
    y = oracle.grid(25)[0]
    sh = (1, 23, 11, 6)
    x = (np.zeros(sh, complex), np.zeros(sh, complex), (u_wall * y)[None].copy(), np.zeros((1, 25)))
    z = ch.step(x, 10)
    assert np.abs(z[2] - x[2]).max() < 1e-14 * abs(u_wall)
    s = ch.stats(z)
    assert abs(s["tau_bottom"][0] - u_wall) < 1e-13 * abs(u_wall)
    assert abs(s["tau_top"][0] - u_wall) < 1e-13 * abs(u_wall)


@pytest.mark.parametrize("q", [2.0, 0.25])
def test_laminar_poiseuille_at_other_fluxes_is_steady(q):
    """At bulk flux Q the laminar profile is U = (3Q/4)(1 - y^2), held by the
    pressure gradient gamma = 3Q/(2 Re) (0 = gamma + U''/Re)."""
    re = 1000.0
    ch = oracle.Channel(16, 25, 16, 2 * np.pi, np.pi, re, 0.005, "poiseuille", bulk_flux=q)
    y = oracle.grid(25)[0]
    sh = (1, 23, 11, 6)
    x = (np.zeros(sh, complex), np.zeros(sh, complex), (0.75 * q * (1 - y ** 2))[None].copy(), np.zeros((1, 25)))
    z = ch.step(x, 10)
    assert np.abs(z[2] - x[2]).max() < 1e-14 * q
    # gamma = (Q - flux0) / flux1 cancels in Q - flux0: relative rounding about
    # eps Q / (flux1 gamma) ~ eps Re / (2 dt) = 2e-11 here
    assert abs(ch.last_gamma[0] - 1.5 * q / re) < 1e-10 * (1.5 * q / re)
    assert abs(ch.stats(z)["bulk_flux"][0] - q) < 1e-14 * max(q, 1.0)


@pytest.mark.parametrize("m", [1, 2])
def test_viscous_streak_decays_by_closed_form_factor(m):
    """A streamwise-uniform streak on laminar Couette has no nonlinear term
    (v = w = 0, d/dx = 0), so one step multiplies eta by the h = 1 CN factor
    (1 + g mu)/(1 - g mu), g = dt/(2 Re); for eta = cos(pi y / 2),
    mu = -(pi/2)^2 - kz^2 (the Dirichlet eigenvalue on [-1, 1])."""
    mx, my, mz, re, dt = 4, 33, 7, 400.0, 0.01
    lx, lz = 2 * np.pi, 1.2 * np.pi
    ch = oracle.Channel(mx, my, mz, lx, lz, re, dt, "couette")
    x = _state(dns_synth.make_state(mx, my, mz, lx, lz, "couette", 1, 0, 0.0))
    v, eta, U, W = (np.array(a) for a in x)
    yi = ch.y[1:-1]
    prof = 1e-3 * np.cos(np.pi * yi / 2)
    eta[0, :, ch.Kz + m, 0] = prof * (0.3 + 0.7j)
    eta[0, :, ch.Kz - m, 0] = prof * (0.3 - 0.7j)
    y = ch.step((v, eta, U, W), 1)
    kz = m * 2 * np.pi / lz
    g = dt / (2 * re)
    mu = -(np.pi / 2) ** 2 - kz ** 2
    fac = (1 + g * mu) / (1 - g * mu)
    assert np.abs(y[1] - fac * eta).max() < 1e-13 * np.abs(eta).max()
    assert np.abs(y[0]).max() == 0.0
    assert np.abs(y[2] - U).max() < 1e-15


def test_orr_sommerfeld_mode_grows_at_linear_rate():
    """An infinitesimal Tollmien-Schlichting wave (Re = 10^4, alpha = 1) in
    Poiseuille flow grows and travels at the published Orr-Sommerfeld rate."""
    g = dict((k, float(v)) for k, v in _read_golden("orr_sommerfeld_re1e4.txt"))
    c_pub = g["c_r"] + 1j * g["c_i"]
    scipy_linalg = pytest.importorskip("scipy.linalg")
    re, dt, my = 1.0e4, 0.01, 81
    ch = oracle.Channel(4, my, 1, 2 * np.pi, 1.0, re, dt, "poiseuille")
    yi = ch.y[1:-1]
    n = my - 2
    # discrete Orr-Sommerfeld eigenproblem on the same D2_int / D4c:
    # i alpha [(U - c)(D2 - a^2) - U''] v = (1/Re)(D2 - a^2)^2 v
    a = 1.0
    I = np.eye(n)
    L = ch.D2[1:-1, 1:-1] - a * a * I
    LL = ch.D4c - 2 * a * a * ch.D2[1:-1, 1:-1] + a ** 4 * I
    U = np.diag(1 - yi ** 2)
    A = 1j * a * (U @ L + 2.0 * I) - LL / re
    B = 1j * a * L
    ev, vec = scipy_linalg.eig(A, B)
    k = np.argmax(ev.imag)
    c_disc = ev[k]
    assert abs(c_disc - c_pub) < 2e-7
    vos = vec[:, k] / vec[np.argmax(np.abs(vec[:, k])), k]
    st = _state(dns_synth.make_state(4, my, 1, 2 * np.pi, 1.0, "poiseuille", 1, 0, 0.0))
    v, eta, Um, W = (np.array(s) for s in st)
    v[0, :, 0, 1] = 1e-9 * vos
    nsteps = 50
    y = ch.step((v, eta, Um, W), nsteps)
    ratio = np.vdot(vos, y[0][0, :, 0, 1]) / np.vdot(vos, v[0, :, 0, 1])
    c_num = 1j * np.log(ratio) / (a * nsteps * dt)
    assert abs(c_num - c_pub) < 2e-6
    assert abs(c_num.imag - c_pub.imag) < 1e-6


# ---------------------------------------------------------- invariants

@pytest.fixture(scope="module")
def couette_small():
    ch = oracle.Channel(16, 33, 16, 1.75 * np.pi, 1.2 * np.pi, 400.0, 0.01, "couette")
    st = dns_synth.make_state(16, 33, 16, 1.75 * np.pi, 1.2 * np.pi, "couette", 2, 1000, 5e-2)
    return ch, _state(st)


def test_divergence_free_and_hermitian(couette_small):
    ch, x = couette_small
    y = ch.step(x, 5)
    s = ch.stats(y)
    assert np.all(s["max_div"] < 1e-14)
    for a in (y[0], y[1]):
        col = a[:, :, :, 0]
        assert np.abs(col - np.conj(col[:, :, ::-1])).max() < 1e-15 * np.abs(col).max() + 1e-300


@pytest.mark.parametrize("flow,mx,my,mz", [("couette", 16, 33, 16), ("poiseuille", 12, 17, 20)])
def test_statistics_equal_physical_space_averages(flow, mx, my, mz):
    """The one-point statistics (Sec. 4) are spectral sums (Parseval, each
    kx > 0 column counted twice for its conjugate); here the same quantities
    are formed the plain way, from the velocity on the physical grid (a library
    inverse FFT): <u'u'>, <v'v'>, <w'w'>, <u'v'> as x-z averages of products of
    the fluctuations about the x-z mean, and the kinetic energies as the
    Clenshaw-Curtis average over y of 1/2 |u|^2 (the wall nodes carry only the
    mean flow)."""
    lx, lz = 2 * np.pi, np.pi
    ch = oracle.Channel(mx, my, mz, lx, lz, 500.0, 0.01, flow)
    x = ch.step(_state(dns_synth.make_state(mx, my, mz, lx, lz, flow, 2, 321, 1e-1)), 2)
    s = ch.stats(x)
    f = ch.velocity(*x)
    phys = {k: ch.to_physical(f[k]) for k in ("u", "v", "w")}        # [e, y, z, x]
    mean = {k: p.mean(axis=(-2, -1)) for k, p in phys.items()}
    assert np.abs(mean["u"] - x[2]).max() < 1e-15 and np.abs(mean["w"] - x[3]).max() < 1e-15
    assert np.abs(mean["v"]).max() < 1e-17
    fl = {k: p - mean[k][..., None, None] for k, p in phys.items()}
    scale = max(np.abs(fl[k]).max() for k in fl) ** 2
    for key, (a, b) in {"uu": ("u", "u"), "vv": ("v", "v"), "ww": ("w", "w"), "uv": ("u", "v")}.items():
        direct = (fl[a] * fl[b]).mean(axis=(-2, -1))
        direct[:, 0] = 0.0
        direct[:, -1] = 0.0
        assert np.abs(s[key] - direct).max() < 1e-13 * scale, key
        assert np.abs(direct).max() > 1e-3 * scale, key    # the check is not vacuous
    w = oracle.cc_weights(my)
    q = sum(fl[k] ** 2 for k in fl).mean(axis=(-2, -1))
    q[:, 0] = 0.0
    q[:, -1] = 0.0
    e_pert = 0.25 * (q @ w)
    e_mean = 0.25 * ((mean["u"] ** 2 + mean["w"] ** 2) @ w)
    assert np.allclose(s["e_pert"], e_pert, rtol=1e-12, atol=0)
    assert np.allclose(s["e_total"], e_pert + e_mean, rtol=1e-13, atol=0)


def test_cfl_of_laminar_profiles_is_the_closed_form():
    """Laminar flows carry only U(y): the CFL number (reading: dt max of
    |u|/dx + |v|/dy + |w|/dz over the interior collocation points) is
    dt max_j |U(y_j)| Mx / Lx over the interior nodes."""
    for flow, prof in (("couette", lambda y: y), ("poiseuille", lambda y: 1.0 - y ** 2)):
        for my in (17, 32):
            mx, mz, lx, lz, dt = 16, 12, 1.75 * np.pi, 1.2 * np.pi, 0.01
            ch = oracle.Channel(mx, my, mz, lx, lz, 400.0, dt, flow)
            x = _state(dns_synth.make_state(mx, my, mz, lx, lz, flow, 1, 0, 0.0))
            y = oracle.grid(my)[0]
            want = dt * np.abs(prof(y[1:-1])).max() * mx / lx
            assert abs(ch.stats(x)["cfl"][0] - want) < 1e-14 * want, (flow, my)


def test_cfl_equals_brute_force_fourier_sums():
    """CFL number of a random state against the velocity summed mode by mode in
    real form, f(x, z) = sum_m Re c(0, m) e^(i kz z) + 2 sum_(n >= 1) sum_m
    Re c(n, m) e^(i (kx x + kz z)), at every interior collocation point."""
    mx, my, mz, lx, lz, dt = 10, 9, 13, 2 * np.pi, np.pi, 0.02
    ch = oracle.Channel(mx, my, mz, lx, lz, 300.0, dt, "poiseuille")
    x = ch.step(_state(dns_synth.make_state(mx, my, mz, lx, lz, "poiseuille", 2, 77, 2e-1)), 1)
    f = ch.velocity(*x)
    Kx, Kz = (mx - 1) // 3, (mz - 1) // 3
    xs = np.arange(mx) * lx / mx
    zs = np.arange(mz) * lz / mz
    y = oracle.grid(my)[0]
    dy = [min(y[j] - y[j - 1], y[j + 1] - y[j]) for j in range(1, my - 1)]
    want = np.zeros(2)
    for e in range(2):
        for j in range(1, my - 1):
            for iz, z in enumerate(zs):
                for ix, xx in enumerate(xs):
                    vals = []
                    for k in ("u", "v", "w"):
                        tot = 0.0
                        for mi in range(2 * Kz + 1):
                            for n in range(Kx + 1):
                                c = f[k][e, j, mi, n]
                                ph = 2 * np.pi * (n * xx / lx + (mi - Kz) * z / lz)
                                term = c.real * np.cos(ph) - c.imag * np.sin(ph)
                                tot += term if n == 0 else 2.0 * term
                        vals.append(abs(tot))
                    r = vals[0] * mx / lx + vals[1] / dy[j - 1] + vals[2] * mz / lz
                    want[e] = max(want[e], dt * r)
    got = ch.stats(x)["cfl"]
    assert np.allclose(got, want, rtol=1e-12, atol=0)
    assert np.all(want > 2 * dt * mx / lx)   # the perturbation dominates the laminar dt Mx / Lx


def test_poiseuille_flux_constant_under_perturbation():
    ch = oracle.Channel(16, 33, 16, 2 * np.pi, np.pi, 1650.0, 0.005, "poiseuille")
    x = _state(dns_synth.make_state(16, 33, 16, 2 * np.pi, np.pi, "poiseuille", 2, 2000, 5e-2,
                                    n_max=4, m_max=4))
    y = ch.step(x, 5)
    assert np.abs(ch.stats(y)["bulk_flux"] - 4.0 / 3.0).max() < 1e-14
    assert np.abs(y[2] - x[2]).max() > 1e-9    # the mean flow did respond


def test_couette_shift_rotate_symmetry_is_preserved():
    """(x, y, z) -> (-x, -y, z), (u, v, w) -> (-u, -v, w) maps plane Couette
    flow onto itself; a symmetric state stays symmetric to round-off."""
    ch = oracle.Channel(10, 25, 10, 1.75 * np.pi, 1.2 * np.pi, 400.0, 0.01, "couette")
    st = dns_synth.make_state(10, 25, 10, 1.75 * np.pi, 1.2 * np.pi, "couette", 1, 7, 5e-2)

    def symm(a):       # x_hat(n, m, y) = -conj x_hat(n, -m, -y)
        return 0.5 * (a - np.conj(a[:, ::-1, ::-1, :]))

    v, eta = symm(st["v"]), symm(st["eta"])
    U = st["U"]
    y = ch.step((v, eta, U, st["W"]), 5)
    for a in (y[0], y[1]):
        assert np.abs(a - symm(a)).max() < 1e-15 * max(1.0, np.abs(a).max()) * 50
    assert np.abs(y[2] + y[2][:, ::-1]).max() < 1e-14
    assert np.abs(y[0]).max() > 1e-4


def test_members_are_independent(couette_small):
    ch, x = couette_small
    both = ch.step(x, 3)
    alone = ch.step(tuple(a[1:2] for a in x), 3)
    for a, b in zip(both, alone):   # BLAS may block differently per batch size
        assert np.abs(a[1:2] - b).max() <= 1e-14 * max(np.abs(b).max(), 1e-300)


def test_energy_budget_residual_is_second_order_in_dt():
    """Kinetic-energy balance of plane Couette flow: dE/dt = wall work -
    dissipation (the advection term only redistributes energy).  The discrete
    residual of the central difference of E falls as O(dt^2) until it meets the
    spatial floor (about 1e-8 here), so dt is taken in 0.08 .. 0.02."""
    mx, my, mz, re = 16, 33, 16, 400.0
    lx, lz = 1.75 * np.pi, 1.2 * np.pi
    st = _state(dns_synth.make_state(mx, my, mz, lx, lz, "couette", 1, 11, 5e-2, n_max=3, m_max=3))
    res = []
    for dt in (0.08, 0.04, 0.02):
        ch = oracle.Channel(mx, my, mz, lx, lz, re, dt, "couette")
        xm = st
        x0 = ch.step(xm, 1)
        xp = ch.step(x0, 1)
        E = [ch.stats(x)["e_total"][0] for x in (xm, x0, xp)]
        s0 = ch.stats(x0)
        dEdt = (E[2] - E[0]) / (2 * dt)
        rhs = s0["wall_work"][0] - s0["dissipation"][0]
        res.append(abs(dEdt - rhs))
        assert abs(dEdt - rhs) < 1e-4 * abs(s0["dissipation"][0])
    assert res[0] / res[1] > 3.5 and res[1] / res[2] > 3.5


# ------------------------------------------- shared-mean (S3T-type) ensemble

def _with_shared_kx0(x):
    """Every member gets the member average of the kx = 0 part (n = 0 column of
    v, eta and the mean profiles U00, W00); the kx != 0 parts stay per member."""
    v, eta, U, W = (np.array(a) for a in x)
    for a in (v, eta):
        a[:, :, :, 0] = a[:, :, :, 0].mean(axis=0)[None]
    U[:] = U.mean(axis=0)[None]
    W[:] = W.mean(axis=0)[None]
    return (v, eta, U, W)


@pytest.fixture(scope="module")
def s3t_small():
    args = (16, 33, 16, 2 * np.pi, 1.2 * np.pi, 1000.0, 0.01, "couette")
    plain = oracle.Channel(*args)
    shared = oracle.Channel(*args, shared_mean=True)
    st = dns_synth.make_state(16, 33, 16, 2 * np.pi, 1.2 * np.pi, "couette", 3, 300, 5e-2)
    return plain, shared, _with_shared_kx0(_state(st))


def test_shared_mean_with_one_member_is_the_plain_step(s3t_small):
    plain, shared, x = s3t_small
    one = tuple(a[1:2] for a in x)
    for a, b in zip(shared.step(one, 3), plain.step(one, 3)):
        assert np.array_equal(a, b)


def test_shared_mean_ensemble_of_copies_is_independent_members(s3t_small):
    plain, shared, x = s3t_small
    copies = tuple(np.repeat(a[1:2], 3, axis=0) for a in x)
    for a, b in zip(shared.step(copies, 3), plain.step(copies, 3)):
        assert np.abs(a - b).max() <= 1e-13 * max(np.abs(b).max(), 1e-300)


def test_shared_mean_kx0_flow_stays_shared_and_moves(s3t_small):
    """The kx = 0 flow of all members stays identical (bit for bit: every member
    receives the same averaged forcing), it is driven away from its start, and
    the kx != 0 parts remain different per member."""
    plain, shared, x = s3t_small
    y = shared.step(x, 4)
    for a in (y[0], y[1]):
        assert np.array_equal(a[0, :, :, 0], a[1, :, :, 0]) and np.array_equal(a[0, :, :, 0], a[2, :, :, 0])
        assert np.abs(a[0, :, :, 1:] - a[1, :, :, 1:]).max() > 1e-6
    assert np.array_equal(y[2][0], y[2][1]) and np.array_equal(y[2][0], y[2][2])
    assert np.abs(y[0][0, :, :, 0] - x[0][0, :, :, 0]).max() > 1e-8
    assert np.abs(y[2][0] - x[2][0]).max() > 1e-8


def test_shared_mean_forcing_and_update_average_the_plain_ones(s3t_small):
    """First sub-step: the shared-mean forcing of the kx = 0 modes (F, G and the
    mean forcings) equals the member average of the plain forcing (the step is
    linear in the nonlinear term), the kx != 0 forcing is the plain one, and by
    linearity of the CN update the shared kx = 0 state after the sub-step is the
    member average of the plain sub-step states."""
    plain, shared, x = s3t_small
    Fp = plain.forcing(x)
    Fs = shared.forcing(x)
    for p, s in zip(Fp[:2], Fs[:2]):
        avg = p[:, :, :, 0].mean(axis=0)
        scale = np.abs(avg).max()
        assert scale > 0
        for e in range(3):
            assert np.abs(s[e, :, :, 0] - avg).max() <= 1e-13 * scale
        assert np.array_equal(s[:, :, :, 1:], p[:, :, :, 1:])
    for p, s in zip(Fp[2:], Fs[2:]):
        avg = p.mean(axis=0)
        assert np.abs(s - avg[None]).max() <= 1e-13 * max(np.abs(avg).max(), 1e-300)
    up = plain.update(x, Fp, 0.5)
    us = shared.update(x, Fs, 0.5)
    for p, s in zip(up[:2], us[:2]):
        avg = p[:, :, :, 0].mean(axis=0)
        assert np.abs(s[:, :, :, 0] - avg[None]).max() <= 1e-13 * np.abs(avg).max()
    for p, s in zip(up[2:], us[2:]):
        assert np.abs(s - p.mean(axis=0)[None]).max() <= 1e-13 * max(np.abs(p).max(), 1e-300)


# ------------------------------------------------ rotational nonlinear form

def test_rotational_form_forcing_equals_advective_where_products_are_resolved():
    """The two forms differ by grad(|u|^2 / 2).  Its curl vanishes: G (x and z
    derivatives only, spectral) agrees to round-off for any state; F also uses
    the Chebyshev collocation derivative in y, which differentiates |u|^2 / 2
    exactly when it is a polynomial of degree <= My - 1 -- true for these
    states (v of degree 8, eta of degree 6 in y, laminar mean: |u|^2 of degree
    16) at My = 33 and 17 but not at My = 13, where F differs at the level of
    the y aliasing."""
    def forcings(form, my):
        ch = oracle.Channel(16, my, 16, 2 * np.pi, np.pi, 800.0, 0.01, "couette", form=form)
        x = _state(dns_synth.make_state(16, my, 16, 2 * np.pi, np.pi, "couette", 2, 4321, 5e-2,
                                        n_max=3, m_max=3))
        return ch.forcing(x)
    adv, rot = forcings("advective", 33), forcings("rotational", 33)
    for a, b in zip(adv, rot):
        scale = max(np.abs(a).max(), 1e-300)
        assert np.abs(a - b).max() <= 1e-12 * scale
    adv, rot = forcings("advective", 17), forcings("rotational", 17)
    for a, b in zip(adv, rot):
        assert np.abs(a - b).max() <= 1e-12 * max(np.abs(a).max(), 1e-300)
    adv, rot = forcings("advective", 13), forcings("rotational", 13)
    G_scale = np.abs(adv[1]).max()
    assert np.abs(adv[1] - rot[1]).max() <= 1e-12 * G_scale             # G: exact for any My
    dF = np.abs(adv[0] - rot[0]).max() / np.abs(adv[0]).max()
    assert 1e-4 < dF < 1e-1                                              # F: y aliasing only
    for a, b in zip(adv[2:], rot[2:]):                                   # mean forcing: same in both
        assert np.array_equal(a, b)


def test_rotational_form_step_stays_divergence_free_and_close_to_advective():
    ch_a = oracle.Channel(16, 33, 16, 1.75 * np.pi, 1.2 * np.pi, 400.0, 0.01, "couette")
    ch_r = oracle.Channel(16, 33, 16, 1.75 * np.pi, 1.2 * np.pi, 400.0, 0.01, "couette", form="rotational")
    x = _state(dns_synth.make_state(16, 33, 16, 1.75 * np.pi, 1.2 * np.pi, "couette", 2, 77, 5e-2))
    ya, yr = ch_a.step(x, 5), ch_r.step(x, 5)
    assert np.all(ch_r.stats(yr)["max_div"] < 1e-14)
    # the states grow in y-degree, so the forms separate slowly (y aliasing)
    for a, b in zip(ya[:2], yr[:2]):
        d = np.abs(a - b).max() / np.abs(a).max()
        assert 1e-12 < d < 1e-5
    for a, b in zip(ya[2:], yr[2:]):      # mean flow (U, W) as one field
        assert np.abs(a - b).max() < 1e-8 * np.abs(ya[2]).max()
