"""Pins of the stochastic-forcing oracle (oracle.forcing): the structures are
eigenvectors of the DNS's discrete diffusion operators (the Stokes-mode and
sine-mode formulas and their transcendental roots are right), they have unit
energy by the DNS oracle's statistics and are mutually orthogonal, the noise
generator is the published SplitMix64 / Box-Muller one (agrees with the
independent input generator and has unit variance), one step from rest gains
dt * eps / sqrt(dt) * sum xi f to first order, and the ensemble-mean energy
gained over a step is the requested injection rate times dt."""
import numpy as np
import pytest

import dns_synth
import oracle
from oracle.forcing import StochasticForcing, normals

pytestmark = pytest.mark.timeout(600)


def _ch(my=33, mz=16, re=1000.0, dt=0.01, flow="couette", u_wall=1.0):
    return oracle.Channel(16, my, mz, 2 * np.pi, np.pi, re, dt, flow, u_wall=u_wall)


@pytest.mark.parametrize("my,n", [(33, 1), (25, 2), (49, 3)])
def test_structures_are_eigenvectors_of_the_discrete_diffusion_operators(my, n):
    ch = _ch(my=my)
    sf = StochasticForcing(ch, n, 4, 1e-3, 1)
    D2 = ch.D2[1:-1, 1:-1]
    I = np.eye(ch.nyi)
    for mi, kz in enumerate(ch.kz):
        k2 = ch.kx[n] ** 2 + kz * kz
        Lap = D2 - k2 * I
        Lv = np.linalg.solve(Lap, ch.D4c - 2 * k2 * D2 + k2 * k2 * I) / ch.re
        for j in range(4):
            for L, b in ((Lv, 0), (Lap / ch.re, 1)):
                f, lam = sf.f[mi, b, j], sf.lam[mi, b, j]
                assert np.abs(L @ f - lam * f).max() < 1e-9 * np.abs(lam * f).max(), (mi, b, j)
        # least damped first, v and eta decay rates interleave with the textbook values
        assert np.all(np.diff(sf.lam[mi, 0]) < 0) and np.all(np.diff(sf.lam[mi, 1]) < 0)
        assert np.isclose(sf.lam[mi, 1, 0], -((np.pi / 2) ** 2 + k2) / ch.re, rtol=1e-15)


def test_structures_have_unit_energy_and_are_orthogonal():
    ch = _ch()
    n = 1
    sf = StochasticForcing(ch, n, 4, 1e-3, 1)
    mi = ch.Kz + 2
    nyi, nm, nk = ch.nyi, 2 * ch.Kz + 1, ch.Kx + 1

    def e_pert(fv, fe):
        v = np.zeros((1, nyi, nm, nk), complex)
        e = np.zeros_like(v)
        v[0, :, mi, n] = fv
        e[0, :, mi, n] = fe
        U = np.zeros((1, ch.my)); W = np.zeros((1, ch.my))
        return ch.stats((v, e, U, W))["e_pert"][0]

    z = np.zeros(nyi)
    for j in range(4):
        # a kx != 0 column of a real field carries the -kx mode too: twice the unit energy
        assert abs(e_pert(sf.f[mi, 0, j], z) - 2.0) < 1e-12
        assert abs(e_pert(z, sf.f[mi, 1, j]) - 2.0) < 1e-12
    for b in (0, 1):
        for i in range(4):
            for j in range(i + 1, 4):
                args = [(sf.f[mi, 0, i] + sf.f[mi, 0, j], z), (z, sf.f[mi, 1, i] + sf.f[mi, 1, j])][b]
                assert abs(e_pert(*args) - 4.0) < 1e-8, (b, i, j)


def test_noise_generator_is_the_published_one_with_unit_variance():
    c = np.arange(200000, dtype=np.uint64)
    a = normals(77, c)
    assert np.array_equal(a, dns_synth.normal(77, c))      # two independent implementations
    assert abs(a.mean()) < 0.01 and abs(a.var() - 1.0) < 0.01
    sf = StochasticForcing(_ch(), 1, 3, 1e-3, 5)
    x = sf.xi(0, 4000)
    assert abs(np.mean(np.abs(x) ** 2) - 1.0) < 0.01 and abs(np.mean(x * x)) < 0.01
    assert not np.array_equal(sf.xi(1, 4)[0], x[0])


def test_one_step_from_rest_gains_the_forcing_increment():
    """Zero base flow, tiny amplitude (the advection term is quadratic, hence
    negligible): after one step v = sqrt(dt) eps sum xi_j f_j and eta likewise,
    to first order in dt (the viscous decay within the step)."""
    ch = _ch(dt=1e-4, u_wall=0.0)
    E, n = 3, 2
    sf = StochasticForcing(ch, n, 4, 1e-10, 9)
    ch.stochastic = sf
    z = np.zeros((E, ch.nyi, 2 * ch.Kz + 1, ch.Kx + 1), complex)
    v, e, U, W = ch.step((z, z.copy(), np.zeros((E, ch.my)), np.zeros((E, ch.my))), 1)
    x = sf.xi(0, E)
    s = np.sqrt(ch.dt) * sf.eps
    want_v = s * np.einsum("emj,mjy->eym", x[:, :, 0], sf.f[:, 0])
    want_e = s * np.einsum("emj,mjy->eym", x[:, :, 1], sf.f[:, 1])
    rel = lambda a, b: np.abs(a - b).max() / np.abs(b).max()
    assert rel(v[:, :, :, n], want_v) < 1e-4 and rel(e[:, :, :, n], want_e) < 1e-4
    # other columns only through the (quadratic, here ~1e-11 relative) self-interaction
    other = np.delete(np.arange(ch.Kx + 1), n)
    assert np.abs(v[:, :, :, other]).max() < 1e-8 * np.abs(want_v).max()
    assert ch.fstep == 1


def test_ensemble_energy_gain_over_a_step_is_the_injection_rate():
    ch = _ch(dt=1e-3, u_wall=0.0)
    E, rate = 48, 1e-6
    ch.stochastic = StochasticForcing(ch, 1, 4, rate, 2024)
    z = np.zeros((E, ch.nyi, 2 * ch.Kz + 1, ch.Kx + 1), complex)
    x = ch.step((z, z.copy(), np.zeros((E, ch.my)), np.zeros((E, ch.my))), 1)
    gain = np.mean(ch.stats(x)["e_pert"]) / ch.dt
    # chi-square scatter: 2 * (11 kz x 2 blocks x 4 structures) real dof per member
    sigma = np.sqrt(2.0 / (E * 2 * 88))
    assert abs(gain / rate - 1.0) < 5 * sigma, (gain / rate, sigma)
