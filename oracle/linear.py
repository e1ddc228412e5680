"""Oracle: linearised forward / adjoint disturbance ensembles about a
streamwise-mean base flow, and the optimal-growth iteration built on them, in
plain numpy FP64.

TEST INFRASTRUCTURE ONLY (like oracle.dns): nothing in the product imports it.

What it follows (paper, "Diagnostic utilities that benefit from
vectorization" and "Growth functional and linearized adjoint equations of
streamwise-mean flow dynamics"):
  * the disturbances have one streamwise wavenumber kx = n (2 pi / Lx), n >= 1,
    and every kept spanwise wavenumber kz = m (2 pi / Lz), |m| <= Kz; the base
    flow B = (U, V, W)(y, z) is streamwise-invariant and frozen;
  * forward equations (linearised Navier-Stokes):
        du'/dt = -[(B . grad) u' + (u' . grad) B] - grad p' + (1/Re) lap u',
    adjoint equations, integrated in reversed time tau = T - t:
        dlam/dtau = (B . grad) lam - (grad B)^T lam - grad b + (1/Re) lap lam,
    ((grad B)^T lam)_j = sum_i lam_i d_j B_i; the paper writes the second term
    as +U_i grad lam_i, which differs from -lam_i grad U_i by the gradient
    grad(U_i lam_i) that the multiplier b absorbs;
  * both are advanced with the DNS's own v-eta CN/RK3 scheme (Sec. 3.1) with the
    single-kx operators: the "nonlinear term" N of the DNS is replaced by
        N_fwd(u') = (B . grad) u' + (u' . grad) B,
        N_adj(lam) = -(B . grad) lam + (grad B)^T lam,
    so that the equation reads d/dt = -N - grad p + (1/Re) lap in both cases;
  * the optimal-growth loop (forward-adjoint iteration of Luchini 2000): the
    adjoint starts from the final forward state, is integrated over the same
    interval, and the set of adjoint results is orthonormalised by Gram-Schmidt
    in the energy inner product to give the next forward initial conditions.

Readings where the paper is silent (each also in the design notes):
  * energy inner product <a, b> = (1/4) sum_m sum_j w_j (conj(u_a) u_b +
    conj(v_a) v_b + conj(w_a) w_b) over the interior Chebyshev nodes (w_j the
    Clenshaw-Curtis weights, walls carry nothing), i.e. the volume average of
    (1/2)|u|^2 for the complex single-harmonic field; with the explicit u, w
    recovery it equals (1/4) sum w_j (conj(v_a) v_b + (conj(Dv_a) Dv_b +
    conj(eta_a) eta_b) / k^2), Dv = D1 applied to v with v = 0 at the walls;
  * Gram-Schmidt is the modified algorithm in member order, each vector
    normalised before it is projected out of the later ones; the growth
    estimate of vector k is its energy norm before normalisation (after a
    forward-adjoint pass that norm approaches sigma_k^2 = G_k);
  * the base flow is given on the physical (y, z) grid (walls included) and is
    truncated to |m| <= Kz before use, so that its products with the
    disturbances are free of aliasing on the 3/2 grid; its y-derivatives are the
    collocation derivative D1 on all My nodes, its z-derivatives spectral;
  * the step dt is the group's own (the paper multiplies the DNS step by a
    factor t_f = 5 for these runs; that is the caller's choice).
Array layout: v[e, j, m + Kz] complex128 (j interior), base arrays [My, Mz].
"""
import numpy as np

from .dns import grid, cc_weights, cn_operators, fundamental, cn_rk3


class Linear:
    """A group of disturbance vectors of one kx about one frozen base flow
    (Sec. 4.1.1, "Diagnostic utilities that benefit from vectorization";
    Appendix B)."""

    def __init__(self, my, mz, lx, lz, re, dt, kx_index, U, V, W):
        assert kx_index >= 1
        self.my, self.mz, self.lx, self.lz, self.re, self.dt = my, mz, lx, lz, re, dt
        self.Kz = (mz - 1) // 3
        self.nyi = my - 2
        self.y, self.D1, self.D2, self.D4c = grid(my)
        self.w = cc_weights(my)
        self.D1i = self.D1[1:-1, 1:-1]
        a1, a3 = fundamental(lx), fundamental(lz)
        self.kx = kx_index * a1
        self.kz = np.arange(-self.Kz, self.Kz + 1) * a3                  # [m + Kz]
        self.k2 = self.kx * self.kx + self.kz * self.kz
        # implicit operators per |m| (single-kx precalculated matrices), per h
        pk2 = np.array([self.kx * self.kx + (am * a3) * (am * a3) for am in range(self.Kz + 1)])
        absm = np.abs(np.arange(-self.Kz, self.Kz + 1))
        self.ops = {}
        for h in (0.5, 1.0):
            self.ops[h] = tuple(a[absm] for a in cn_operators(my, pk2, dt, re, h))
        self.adjoint = False
        self.set_base(U, V, W)

    # ------------------------------------------------------------ base flow
    def _to_phys(self, c):
        """Kept coefficients [..., 2Kz+1] -> values on the Mz points (inverse
        transform, unnormalised, zero padded)."""
        Kz = self.Kz
        Z = np.zeros(c.shape[:-1] + (self.mz,), dtype=np.complex128)
        Z[..., :Kz + 1] = c[..., Kz:]
        if Kz > 0:
            Z[..., self.mz - Kz:] = c[..., :Kz]
        return np.fft.ifft(Z, axis=-1, norm="forward")

    def _to_spec(self, f):
        """Values on the Mz points -> coefficients of the kept kz (forward
        transform carries 1/Mz)."""
        Kz = self.Kz
        F = np.fft.fft(f, axis=-1, norm="forward")
        out = np.zeros(f.shape[:-1] + (2 * Kz + 1,), dtype=np.complex128)
        out[..., Kz:] = F[..., :Kz + 1]
        if Kz > 0:
            out[..., :Kz] = F[..., self.mz - Kz:]
        return out

    def set_base(self, U, V, W):
        """Base flow on the (My, Mz) grid -> nine real fields on the interior
        planes: B_i, d_y B_i, d_z B_i for B = (U, V, W) (Sec. 4.1.1)."""
        self.base = {}
        ikz = 1j * self.kz
        for name, f in (("U", U), ("V", V), ("W", W)):
            c = self._to_spec(np.asarray(f, dtype=np.float64))           # [My, 2Kz+1]
            val = np.real(self._to_phys(c))                              # truncated, [My, Mz]
            dy = self.D1 @ val
            dz = np.real(self._to_phys(ikz[None, :] * c))
            self.base[name] = val[1:-1]
            self.base[name + "y"] = dy[1:-1]
            self.base[name + "z"] = dz[1:-1]

    # ------------------------------------------------------- velocity field
    def velocity(self, v, eta):
        """u, v, w and their y- and z-derivatives on all My nodes, spectral
        [e, My, 2Kz+1] (x-derivatives are i kx times the field; u, w recovered as
        in Sec. 3.2)."""
        E = v.shape[0]
        sh = (E, self.my, 2 * self.Kz + 1)
        vf = np.zeros(sh, dtype=np.complex128); vf[:, 1:-1] = v
        ef = np.zeros(sh, dtype=np.complex128); ef[:, 1:-1] = eta
        Dv = np.einsum("ij,ejm->eim", self.D1, vf)
        D2v = np.einsum("ij,ejm->eim", self.D2, vf)
        De = np.einsum("ij,ejm->eim", self.D1, ef)
        ikx = 1j * self.kx
        ikz = 1j * self.kz[None, None, :]
        k2 = self.k2[None, None, :]
        u = (ikx * Dv - ikz * ef) / k2
        w = (ikz * Dv + ikx * ef) / k2
        uy = (ikx * D2v - ikz * De) / k2
        wy = (ikz * D2v + ikx * De) / k2
        return {"u": u, "v": vf, "w": w, "uy": uy, "vy": Dv, "wy": wy,
                "uz": ikz * u, "vz": ikz * vf, "wz": ikz * w}

    # --------------------------------------------------------- linear terms
    def term(self, v, eta, adjoint=None):
        """N_fwd or N_adj (module docstring) on the interior planes, transformed
        and truncated: three spectral arrays [e, Ny_i, 2Kz+1] (Appendix B)."""
        if adjoint is None:
            adjoint = self.adjoint
        f = self.velocity(v, eta)
        p = {k: self._to_phys(a[:, 1:-1]) for k, a in f.items()}
        B = self.base
        ikx = 1j * self.kx
        comp = (("u", "uy", "uz"), ("v", "vy", "vz"), ("w", "wy", "wz"))
        # (B . grad) a_i = i kx U a_i + V d_y a_i + W d_z a_i
        adv = [ikx * B["U"] * p[a] + B["V"] * p[ay] + B["W"] * p[az] for a, ay, az in comp]
        if not adjoint:
            # + (u' . grad) B_i = v' d_y B_i + w' d_z B_i
            N = [adv[i] + p["v"] * B[c + "y"] + p["w"] * B[c + "z"] for i, c in enumerate("UVW")]
        else:
            # - (B . grad) lam_i + sum_k lam_k d_i B_k (no x-derivative of B)
            N = [-adv[0],
                 -adv[1] + p["u"] * B["Uy"] + p["v"] * B["Vy"] + p["w"] * B["Wy"],
                 -adv[2] + p["u"] * B["Uz"] + p["v"] * B["Vz"] + p["w"] * B["Wz"]]
        return tuple(self._to_spec(a) for a in N)

    def forcing(self, state):
        """F, G of the v-eta equations (Sec. 3.1) from the linear term."""
        v, eta = state
        Nu, Nv, Nw = self.term(v, eta)
        ikx = 1j * self.kx
        ikz = 1j * self.kz[None, None, :]
        phi = ikx * Nu + ikz * Nw
        F = -self.k2[None, None, :] * Nv - np.einsum("ij,ejm->eim", self.D1i, phi)
        G = ikz * Nu - ikx * Nw
        return (F, G)

    def update(self, state_t, Ft, h, s=None):
        """CN sub-step from the state at t with the single-kx operators
        (Eqs. CN1, CN2, valid for the adjoint equations too, Sec. 4.1.1)."""
        v, eta = state_t
        F, G = Ft
        Mv, Pv, Me, Pe = self.ops[h]
        vn = np.einsum("mij,ejm->eim", Mv, v) + np.einsum("mij,ejm->eim", Pv, F)
        en = np.einsum("mij,ejm->eim", Me, eta) + np.einsum("mij,ejm->eim", Pe, G)
        return (vn, en)

    def step(self, state, nsteps=1, adjoint=False):
        """Advance (v, eta) by nsteps CN/RK3 steps of the forward (or adjoint)
        equations (the scheme of Sec. 3.1, as Sec. 4.1.1 applies it)."""
        self.adjoint = adjoint
        x = tuple(np.array(a) for a in state)
        for _ in range(nsteps):
            x = cn_rk3(x, self.forcing, self.update)
        return x

    # ------------------------------------------------------------ energy
    def inner(self, a, b):
        """Energy inner products <a_i, b_j> (module docstring): [Ea, Eb] (Appendix B)."""
        va, ea = a
        vb, eb = b
        Dva = np.einsum("ij,ejm->eim", self.D1i, va)
        Dvb = np.einsum("ij,ejm->eim", self.D1i, vb)
        w = self.w[1:-1]
        ik2 = 1.0 / self.k2
        g = np.einsum("ajm,bjm,j->ab", np.conj(va), vb, w)
        g = g + np.einsum("ajm,bjm,j,m->ab", np.conj(Dva), Dvb, w, ik2)
        g = g + np.einsum("ajm,bjm,j,m->ab", np.conj(ea), eb, w, ik2)
        return 0.25 * g

    def energy(self, state):
        """Energy of every vector: the diagonal of inner (Appendix B)."""
        return np.real(np.diagonal(self.inner(state, state))).copy()

    def orthonormalize(self, state):
        """Modified Gram-Schmidt in the energy inner product, in member order
        (Sec. 4.1.1: the orthonormalisation step).  Returns the orthonormal set
        and each vector's norm before its normalisation."""
        v = np.array(state[0]); eta = np.array(state[1])
        E = v.shape[0]
        r = np.zeros(E)
        for k in range(E):
            xk = (v[k:k + 1], eta[k:k + 1])
            r[k] = np.sqrt(np.real(self.inner(xk, xk)[0, 0]))
            v[k] /= r[k]
            eta[k] /= r[k]
            for j in range(k + 1, E):
                c = self.inner((v[k:k + 1], eta[k:k + 1]), (v[j:j + 1], eta[j:j + 1]))[0, 0]
                v[j] -= c * v[k]
                eta[j] -= c * eta[k]
        return (v, eta), r

    def sweep(self, state, nsteps):
        """One forward-adjoint iteration over nsteps steps each way, followed by
        Gram-Schmidt (Sec. 4.1.1: the forward-adjoint iteration loop).  Returns the next initial conditions and the growth
        estimates (the norms before normalisation)."""
        fwd = self.step(state, nsteps, adjoint=False)
        adj = self.step(fwd, nsteps, adjoint=True)
        self.adjoint = False
        return self.orthonormalize(adj)
