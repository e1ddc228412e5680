"""Oracle: stochastic forcing from eigenvectors of the diffusion operator (the
paper's S3T ensemble run, Sec. "Ensemble integrations": forcing realisations
formed by mixing eigenvectors of the diffusion operator acting on a
(Delta v, eta) state, scaled to equal diffusion rate, at one streamwise
wavenumber).  Plain numpy FP64.

TEST INFRASTRUCTURE ONLY (like oracle.dns): nothing in the product imports it.

Readings (the paper gives the forcing in two sentences; each also in the
design notes):
  * forced modes: one streamwise index n_f (the paper: kx / a = 1) and every
    kept kz; per kz the n_eig least-damped eigenfunctions of each block of the
    diffusion operator on (Delta v, eta), i.e. of d/dt Delta v = Delta Delta v / Re
    with v = Dv = 0 and of d/dt eta = Delta eta / Re with eta = 0 at the walls
    (Delta = D^2 - k^2, k^2 = kx^2 + kz^2):
      v: the Stokes modes, even  phi = cos(mu y) / cos(mu) - cosh(k y) / cosh(k),
                                 mu tan(mu) = -k tanh(k),
                           odd   phi = sin(mu y) / sin(mu) - sinh(k y) / sinh(k),
                                 mu cot(mu) = k coth(k),
         decay rate (mu^2 + k^2) / Re, ordered by increasing mu (even roots in
         ((n - 1/2) pi, n pi), odd roots in (n pi, (n + 1/2) pi), n >= 1);
      eta: sin(j pi (y + 1) / 2), decay rate ((j pi / 2)^2 + k^2) / Re, j >= 1;
    sampled at the interior Chebyshev nodes.  For resolved modes they satisfy
    the eigen-relations of the DNS's own collocation operators (Delta^-1 of the
    clamped Delta Delta, and Delta) to round-off; taking eigenvectors of the
    symmetric part of those operators in energy coordinates instead gives
    spurious growing ones (the clamped fourth derivative is far from
    self-adjoint in the energy norm);
  * "scaled to equal diffusion rate": every structure is scaled to unit
    energy (the statistics' inner product, (1/4) sum_j w_j (|u|^2 + |v|^2 +
    |w|^2) per complex kx column), so under white noise of equal intensity each
    injects energy at the same rate and, at statistical equilibrium,
    dissipates it at that rate;
  * time dependence: complex white noise, one independent realisation per step,
    member, kz and structure, held constant over the three sub-steps of the
    step (their combination weights sum to one, so the step receives it once):
    over a step the state gains dt * eps / sqrt(dt) * sum_j xi_j f_j with
    E|xi_j|^2 = 1;
  * amplitude: the caller's injection rate r of the perturbation energy the
    statistics report (e_pert, which counts the +-kx pair of a real field):
    eps^2 = r / (2 * (number of structures per member));
  * random numbers: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) on counters,
    53-bit uniforms on (0, 1), Box-Muller (cosine branch) from draws 2k, 2k+1;
    xi = (N(c) + i N(c + 1)) / sqrt(2) with
    c = 2 * ((((step * E + member) * (2 Kz + 1) + m_index) * 2 + block) * n_eig + j).
The forcing enters the DNS through its right-hand sides: F (the Delta v
equation's, which the update applies with -h dt A^-1) gains -Delta f_v, and G
gains -f_eta.
"""
import numpy as np

_M64 = 0xFFFFFFFFFFFFFFFF


def _mix64(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def _uniform(seed, k):
    k = np.asarray(k, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _M64) * np.uint64(0xD1342543DE82EF95) + (k + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)
    z = _mix64(z)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normals(seed, counters):
    """Standard normals N(c): Box-Muller (Box and Muller 1958; cosine branch)
    of draws 2c, 2c + 1."""
    c = np.asarray(counters, dtype=np.uint64)
    u1 = _uniform(seed, np.uint64(2) * c)
    u2 = _uniform(seed, np.uint64(2) * c + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def _root(f, lo, hi):
    """Root of f in (lo, hi) where f changes sign (scipy's Brent method)."""
    import scipy.optimize
    return scipy.optimize.brentq(f, lo, hi, xtol=1e-15, rtol=4 * np.finfo(float).eps, maxiter=500)


def stokes_mu(k, count):
    """The first `count` Stokes-mode wavenumbers mu (increasing), with parity:
    eigenfunctions of the diffusion operator that the S3T run of Sec. 4.1
    draws its forcing from."""
    out = []
    n = 1
    while len(out) < count:
        a, b = (n - 0.5) * np.pi, n * np.pi               # even: mu tan mu + k tanh k = 0
        out.append((_root(lambda m: m * np.sin(m) + k * np.tanh(k) * np.cos(m), a + 1e-12, b - 1e-12), 0))
        a, b = n * np.pi, (n + 0.5) * np.pi                  # odd: mu cos mu - k coth k sin mu = 0
        out.append((_root(lambda m: m * np.cos(m) - k / np.tanh(k) * np.sin(m), a + 1e-12, b - 1e-12), 1))
        n += 1
    return out[:count]


class StochasticForcing:
    """Forcing structures of one DNS group (oracle.Channel) and the per-step
    noise they are mixed with (Sec. 4.1, the S3T run)."""

    def __init__(self, ch, kx_index, n_eig, rate, seed):
        assert 1 <= kx_index <= ch.Kx and 1 <= n_eig <= ch.nyi
        self.ch, self.n, self.n_eig, self.rate, self.seed = ch, kx_index, n_eig, rate, seed
        ny = ch.nyi
        D2 = ch.D2[1:-1, 1:-1]
        w = ch.w[1:-1]
        y = ch.y[1:-1]
        kx = ch.kx[kx_index]
        nm = 2 * ch.Kz + 1
        self.lam = np.zeros((nm, 2, n_eig))
        self.f = np.zeros((nm, 2, n_eig, ny))          # structures: block 0 v, block 1 eta
        self.rhs = np.zeros((nm, 2, n_eig, ny))        # their F (block 0) or G (block 1) terms
        for mi, kz in enumerate(ch.kz):
            k2 = kx * kx + kz * kz
            k = np.sqrt(k2)
            Lap = D2 - k2 * np.eye(ny)
            for j, (mu, odd) in enumerate(stokes_mu(k, n_eig)):
                if odd:
                    phi = np.sin(mu * y) / np.sin(mu) - np.sinh(k * y) / np.sinh(k)
                else:
                    phi = np.cos(mu * y) / np.cos(mu) - np.cosh(k * y) / np.cosh(k)
                Dphi = ch.D1i @ phi
                e = 0.25 * (np.sum(w * phi * phi) + np.sum(w * Dphi * Dphi) / k2)
                phi = phi / np.sqrt(e)
                self.lam[mi, 0, j] = -(mu * mu + k2) / ch.re
                self.f[mi, 0, j] = phi
                self.rhs[mi, 0, j] = -(Lap @ phi)
            for j in range(n_eig):
                a = 0.5 * (j + 1) * np.pi
                psi = np.sin(a * (y + 1.0))
                e = 0.25 * np.sum(w * psi * psi) / k2
                psi = psi / np.sqrt(e)
                self.lam[mi, 1, j] = -(a * a + k2) / ch.re
                self.f[mi, 1, j] = psi
                self.rhs[mi, 1, j] = -psi
        self.eps = np.sqrt(rate / (2.0 * (nm * 2 * n_eig)))

    def xi(self, step, E):
        """Complex unit-variance noise [E, 2Kz+1, 2, n_eig] of one step (Sec. 4.1)."""
        nm = 2 * self.ch.Kz + 1
        idx = np.arange(E * nm * 2 * self.n_eig, dtype=np.uint64) + np.uint64(step * E * nm * 2 * self.n_eig)
        c = np.uint64(2) * idx
        z = (normals(self.seed, c) + 1j * normals(self.seed, c + np.uint64(1))) / np.sqrt(2.0)
        return z.reshape(E, nm, 2, self.n_eig)

    def terms(self, step, E):
        """(F_noise, G_noise) [E, Ny, 2Kz+1] at column kx_index for one step:
        the forcing constant over the step, eps / sqrt(dt) sum_j xi_j (rhs_j) (Sec. 4.1)."""
        x = self.xi(step, E)
        s = self.eps / np.sqrt(self.ch.dt)
        Fn = s * np.einsum("emj,mjy->eym", x[:, :, 0], self.rhs[:, 0])
        Gn = s * np.einsum("emj,mjy->eym", x[:, :, 1], self.rhs[:, 1])
        return Fn, Gn
