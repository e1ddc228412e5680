"""Pins of the linearised forward / adjoint oracle (oracle.linear) against
things other than itself: the DNS oracle's advection term (the linear term is
its exact cross term), integration by parts (the adjoint term is the L2
adjoint of the forward term on fields the quadrature integrates exactly),
Parseval and the DNS statistics (energy), a library QR (Gram-Schmidt), and the
matrix exponential of the textbook Orr-Sommerfeld-Squire operator (optimal
growth about laminar Poiseuille flow)."""
import numpy as np
import pytest
import scipy.linalg

import dns_synth
import oracle
from oracle.linear import Linear

pytestmark = pytest.mark.timeout(600)


def _lin(my=25, mz=16, lx=2 * np.pi, lz=np.pi, re=1000.0, dt=0.01, n=2, flow="couette", seed=5,
         streak=0.2, roll=0.02):
    b = dns_synth.make_base_flow(my, mz, lz, flow, seed, streak=streak, roll=roll)
    return Linear(my, mz, lx, lz, re, dt, n, b["U"], b["V"], b["W"]), b


def _dns_state(ch, base, col, dist):
    """A DNS state holding the streamwise-mean base flow in its kx = 0 column and
    the disturbance `dist` in column `col` (E members)."""
    Kz, my = ch.Kz, ch.my
    E = dist["v"].shape[0]
    v = np.zeros((E, my - 2, 2 * Kz + 1, ch.Kx + 1), dtype=np.complex128)
    eta = np.zeros_like(v)

    def spec(f):
        F = np.fft.fft(f, axis=-1, norm="forward")
        out = np.zeros(f.shape[:-1] + (2 * Kz + 1,), dtype=np.complex128)
        out[..., Kz:] = F[..., :Kz + 1]
        out[..., :Kz] = F[..., ch.mz - Kz:]
        return out

    Uh, Vh = spec(base["U"]), spec(base["V"])
    ikz = 1j * ch.kz
    # kx = 0: v = V, eta = dz U - dx W = i kz U; U00, W00 are the m = 0 coefficients
    v[:, :, :, 0] = Vh[None, 1:-1]
    eta[:, :, :, 0] = (ikz[None, :] * Uh)[None, 1:-1]
    v[:, :, Kz, 0] = 0.0
    eta[:, :, Kz, 0] = 0.0
    U00 = np.tile(np.real(Uh[:, Kz]), (E, 1))
    W00 = np.tile(np.real(spec(base["W"])[:, Kz]), (E, 1))
    v[:, :, :, col] = dist["v"]
    eta[:, :, :, col] = dist["eta"]
    return v, eta, U00, W00


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("flow,n", [("couette", 1), ("couette", 2), ("poiseuille", 3)])
def test_forward_term_is_the_cross_term_of_the_advection_term(flow, n):
    """u . grad u is quadratic, so (N(B + u') - N(B - u')) / 2 is exactly
    (B . grad) u' + (u' . grad) B: column n of the DNS oracle's advection term
    about the base flow equals the linear oracle's forward term."""
    my, mz, mx = 25, 16, 16
    lin, base = _lin(my=my, mz=mz, n=n, flow=flow)
    ch = oracle.Channel(mx, my, mz, 2 * np.pi, np.pi, 1000.0, 0.01, flow)
    dist = dns_synth.make_disturbances(my, mz, np.pi, 2, 40 + n)
    vp, ep, U, W = _dns_state(ch, base, n, dist)
    vm, em, _, _ = _dns_state(ch, base, n, {k: -a for k, a in dist.items()})
    Np = ch.nonlinear(vp, ep, U, W)[:3]
    Nm = ch.nonlinear(vm, em, U, W)[:3]
    got = lin.term(dist["v"], dist["eta"], adjoint=False)
    for a, b, c in zip(Np, Nm, got):
        cross = 0.5 * (a[:, :, :, n] - b[:, :, :, n])
        assert _rel(c, cross) < 1e-12


def test_adjoint_term_is_the_l2_adjoint_of_the_forward_term():
    """<lam, N_fwd(u)> = <N_adj(lam), u> in the L2 inner product of the
    primitive velocities (the integration by parts the adjoint is derived by),
    exact here because every integrand is a polynomial of degree < My - 1 and
    the base flow is divergence-free and band-limited."""
    my, mz = 33, 16
    lin, _ = _lin(my=my, mz=mz, n=1, flow="poiseuille")
    u = dns_synth.make_disturbances(my, mz, np.pi, 1, 70)
    lam = dns_synth.make_disturbances(my, mz, np.pi, 1, 71)
    w = lin.w[1:-1]

    def l2(a, b):
        # sum over components, kz and interior nodes (all fields vanish at the walls)
        return sum(np.einsum("ejm,ejm,j->", np.conj(x), y_, w) for x, y_ in zip(a, b))

    fu = lin.velocity(u["v"], u["eta"])
    fl = lin.velocity(lam["v"], lam["eta"])
    prim_u = [fu[c][:, 1:-1] for c in "uvw"]
    prim_l = [fl[c][:, 1:-1] for c in "uvw"]
    Nf = lin.term(u["v"], u["eta"], adjoint=False)
    Na = lin.term(lam["v"], lam["eta"], adjoint=True)
    lhs = l2(prim_l, Nf)
    rhs = l2(Na, prim_u)
    assert abs(lhs) > 1e-3
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # not a tautology: the forward term is not self-adjoint
    Nf_l = lin.term(lam["v"], lam["eta"], adjoint=False)
    assert abs(l2(Nf_l, prim_u) - lhs) > 1e-3 * abs(lhs)


def test_energy_inner_product_is_the_volume_average_and_matches_the_dns_statistics():
    my, mz, n = 25, 16, 2
    lin, base = _lin(my=my, mz=mz, n=n)
    d = dns_synth.make_disturbances(my, mz, np.pi, 3, 11)
    E = lin.energy((d["v"], d["eta"]))
    # Parseval: (1/4) sum_j w_j mean_z (|u|^2 + |v|^2 + |w|^2) of the complex field
    f = lin.velocity(d["v"], d["eta"])
    phys = [lin._to_phys(f[c][:, 1:-1]) for c in "uvw"]
    ms = sum(np.mean(np.abs(p) ** 2, axis=-1) for p in phys)
    assert np.allclose(E, 0.25 * ms @ lin.w[1:-1], rtol=1e-13, atol=0)
    # the DNS statistics count a kx != 0 column twice (the real field carries -kx)
    ch = oracle.Channel(16, my, mz, 2 * np.pi, np.pi, 1000.0, 0.01, "couette")
    zero = {k: np.zeros_like(a) for k, a in base.items()}
    v, eta, U, W = _dns_state(ch, zero, n, d)
    st = ch.stats((v, eta, U, W))
    assert np.allclose(E, 0.5 * st["e_pert"], rtol=1e-13, atol=0)
    G = lin.inner((d["v"], d["eta"]), (d["v"], d["eta"]))
    assert np.allclose(G, np.conj(G.T), rtol=0, atol=1e-14 * np.abs(G).max())


def test_gram_schmidt_is_a_qr_factorisation_in_the_energy_norm():
    my, mz = 25, 16
    lin, _ = _lin(my=my, mz=mz, n=1)
    d = dns_synth.make_disturbances(my, mz, np.pi, 5, 21)
    # make the set ill-conditioned: vector 3 nearly a combination of 0 and 1
    d["v"][3] = d["v"][0] - 0.5j * d["v"][1] + 1e-3 * d["v"][3]
    d["eta"][3] = d["eta"][0] - 0.5j * d["eta"][1] + 1e-3 * d["eta"][3]
    X = (d["v"], d["eta"])
    Q, r = lin.orthonormalize(X)
    G = lin.inner(Q, Q)
    assert np.max(np.abs(G - np.eye(5))) < 1e-12
    C = lin.inner(Q, X)                      # C[k, j] = <q_k, x_j>
    assert np.max(np.abs(np.tril(C, -1))) < 1e-12 * np.abs(C).max()
    # rounding in r_k scales with |x_k|, not with r_k (vector 3 loses 3 digits)
    xn = np.sqrt(lin.energy(X))
    assert np.all(np.abs(np.diag(C) - r) < 1e-12 * xn)
    rec_v = np.einsum("kj,kym->jym", np.triu(C), Q[0])
    assert _rel(rec_v, X[0]) < 1e-12
    # library QR of the energy coordinates (sqrt-weighted v, Dv / k, eta / k)
    w = np.sqrt(0.25 * lin.w[1:-1])[None, :, None]
    ik = 1.0 / np.sqrt(lin.k2)[None, None, :]
    Dv = np.einsum("ij,ejm->eim", lin.D1i, X[0])
    Z = np.concatenate([(w * X[0]).reshape(5, -1), (w * ik * Dv).reshape(5, -1),
                        (w * ik * X[1]).reshape(5, -1)], axis=1).T
    R = np.linalg.qr(Z, mode="r")
    assert np.all(np.abs(np.abs(np.diag(R)) - r) < 1e-12 * xn)


def _oss_gains(my, lz, kz_index, T, re):
    """Energy gains (squared singular values) over [0, T] of the semi-discrete
    Orr-Sommerfeld / Squire operator about laminar Poiseuille flow U = 1 - y^2
    (textbook form, e.g. Schmid & Henningson, Stability and Transition in Shear
    Flows, Sec. 3.1), kx = 1, one kz, from the matrix exponential."""
    b = dns_synth.make_base_flow(my, 8, lz, "poiseuille", 1, streak=0.0, roll=0.0)
    lin = Linear(my, 8, 2 * np.pi, lz, re, 0.01, 1, b["U"], b["V"], b["W"])
    y = lin.y[1:-1]
    U, dU, d2U = 1 - y ** 2, -2 * y, -2 * np.ones_like(y)
    D2, D4, D1 = lin.D2[1:-1, 1:-1], lin.D4c, lin.D1i
    n = lin.nyi
    I = np.eye(n)
    Z = np.zeros((n, n))
    w = lin.w[1:-1]
    kx, kz = lin.kx, lin.kz[lin.Kz + kz_index]
    k2 = kx * kx + kz * kz
    Lap = D2 - k2 * I
    LL = D4 - 2 * k2 * D2 + k2 * k2 * I
    Lvv = np.linalg.solve(Lap, -1j * kx * np.diag(U) @ Lap + 1j * kx * np.diag(d2U) + LL / re)
    L = np.block([[Lvv, Z], [-1j * kz * np.diag(dU), -1j * kx * np.diag(U) + Lap / re]])
    Q = 0.25 * np.block([[np.diag(w) + D1.T @ np.diag(w) @ D1 / k2, Z], [Z, np.diag(w) / k2]])
    C = np.linalg.cholesky(Q).conj().T           # Q = C^H C
    P = C @ scipy.linalg.expm(L * T) @ np.linalg.inv(C)
    return np.linalg.svd(P, compute_uv=False) ** 2


@pytest.mark.parametrize("kz_index", [0, 1])
def test_forward_adjoint_iteration_about_laminar_poiseuille_finds_the_optimal_gains(kz_index):
    """About laminar Poiseuille flow the kz modes decouple, so an iteration
    started in one kz stays there; forward-adjoint sweeps with Gram-Schmidt must
    converge to the leading energy gains of that kz, computed independently from
    the matrix exponential of the Orr-Sommerfeld-Squire operator on a finer grid
    (My = 97; on coarse grids the discrete operator's SVD has spurious
    under-resolved optima that the time-stepped adjoint does not reproduce).
    kz = 0 exercises the Orr-Sommerfeld part; kz != 0 the lift-up coupling
    v -> eta, where the two leading gains nearly coincide and the converged
    quantity is their product (the 2 x 2 subspace's determinant)."""
    my, mz, lz, re, T, dt = 33, 8, np.pi, 1000.0, 2.0, 0.04
    ref = _oss_gains(97, lz, kz_index, T, re)
    b = dns_synth.make_base_flow(my, mz, lz, "poiseuille", 1, streak=0.0, roll=0.0)
    lin = Linear(my, mz, 2 * np.pi, lz, re, dt, 1, b["U"], b["V"], b["W"])
    d = dns_synth.make_disturbances(my, mz, lz, 2, 3)
    mi = lin.Kz + kz_index
    for a in (d["v"], d["eta"]):
        keep = a[:, :, mi].copy()
        a[:] = 0.0
        a[:, :, mi] = keep
    X, _ = lin.orthonormalize((d["v"], d["eta"]))
    for _ in range(30):
        X, r = lin.sweep(X, int(round(T / dt)))
    if kz_index == 0:
        assert np.all(np.abs(r - ref[:2]) < 2e-5 * ref[:2]), (r, ref[:3])
    else:
        assert abs(r[0] * r[1] - ref[0] * ref[1]) < 5e-5 * ref[0] * ref[1], (r, ref[:3])
    # the set stays in the started kz and stays orthonormal
    assert np.max(np.abs(np.delete(X[0], mi, axis=2))) == 0.0
    assert np.max(np.abs(lin.inner(X, X) - np.eye(2))) < 1e-12
