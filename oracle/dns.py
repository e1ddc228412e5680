"""Oracle: one CN/RK3 step of the ensemble v-eta channel DNS, in plain numpy FP64.

TEST INFRASTRUCTURE ONLY.  Nothing in the product imports this module; only the
tests, the smoke check and the benchmark's CPU-baseline leg do.  It is written
to be read against the paper, not to be fast: every array is full size, every
sum is a numpy library call (matmul, FFT) with no blocking or fusion.

Notation (paper Sec. 2-3):
  y_j  flipped Chebyshev-Gauss-Lobatto nodes, j = 0..My-1 (walls at j = 0, My-1)
  kx = n * (2 pi / Lx), n = 0..Kx;  kz = m * (2 pi / Lz), m = -Kz..Kz;
  Kx = (Mx-1)//3, Kz = (Mz-1)//3 (2/3-rule truncation, Sec. 3.2)
  state per member: v_hat, eta_hat on the My-2 interior nodes for every kept
  (n, m) != (0, 0) (zero at (0, 0)); U00, W00 on all My nodes.
Array layout: v[e, j, m + Kz, n] complex128 (j interior), U[e, j] float64.

Readings of the paper where it is silent or garbled (each also in the design notes):
  * kept modes: |n| <= (Mx-1)//3, |m| <= (Mz-1)//3;
  * D2_int = D2 with the first and last rows and columns removed;
  * Delta Delta = D4c - 2 k^2 D2_int + k^4 I (D2_int in the middle term);
  * u, w recovery uses the explicit solutions u = (i kx Dv - i kz eta)/k^2,
    w = (i kz Dv + i kx eta)/k^2 (eta = dz u - dx w);
  * the nonlinear terms are evaluated on the interior planes only and are
    taken as zero on the walls (no slip), where the y-derivative of
    phi = i kx Nu + i kz Nw needs them;
  * the Poiseuille pressure gradient gamma is chosen at every sub-step so that
    the Clenshaw-Curtis integral of U00 equals the prescribed bulk flux;
  * transform convention: forward = sum / (Mx Mz), inverse unnormalised;
  * CFL number (the paper steps at fixed dt and defines none): dt times the
    maximum over the interior collocation points (the Mx x Mz grid of every
    interior plane) of |u|/dx + |v|/dy_j + |w|/dz, mean flow included, with
    dx = Lx/Mx, dz = Lz/Mz and dy_j the smaller of the node's two gaps.
"""
import ctypes
import numpy as np

from . import build as _build

_lib = None


def _ops():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.orc_grid.argtypes = [ctypes.c_int, dp, dp, dp, dp]
        lib.orc_cc_weights.argtypes = [ctypes.c_int, dp]
        lib.orc_cn_ops.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, dp, dp, dp, dp]
        lib.orc_mean_ops.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, dp, dp, dp, dp]
        lib.orc_solve.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp, dp]
        lib.orc_fundamental.argtypes = [ctypes.c_double]
        lib.orc_fundamental.restype = ctypes.c_double
        _lib = lib
    return _lib


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def grid(My):
    """Nodes, D1, D2 = D1 D1 on all My nodes and the clamped D4c (interior):
    the Chebyshev collocation of Sec. 3.2 (the Laplacians of Listing 1 are
    built from them; D4c enters the v operator of Eq. CN1)."""
    y = np.zeros(My); D1 = np.zeros((My, My)); D2 = np.zeros((My, My))
    D4c = np.zeros((My - 2, My - 2))
    rc = _ops().orc_grid(My, _p(y), _p(D1), _p(D2), _p(D4c))
    assert rc == 0
    return y, D1, D2, D4c


def cc_weights(My):
    """Clenshaw-Curtis weights of the nodes: the y-integrals of the bulk flux
    (the constant-flux condition of Sec. 3.2) and of the statistics (Sec. 4)."""
    w = np.zeros(My)
    assert _ops().orc_cc_weights(My, _p(w)) == 0
    return w


def cn_operators(My, k2, dt, re, h):
    """Mv, Pv, Me, Pe for each k^2 in k2 (Eqs. CN1, CN2): arrays [len(k2), n, n]."""
    k2 = np.ascontiguousarray(np.asarray(k2, dtype=np.float64).ravel())
    n = My - 2
    out = [np.zeros((len(k2), n, n)) for _ in range(4)]
    rc = _ops().orc_cn_ops(My, len(k2), _p(k2), dt, re, h, *[_p(a) for a in out])
    assert rc == 0
    return out


def mean_operators(My, dt, re, h):
    """MU, PU, bU (wall terms) and the unit pressure-gradient response Ug of
    the mean-flow update (Eqs. CN3, CN4, Sec. 3.2), built in binary128."""
    n = My - 2
    MU = np.zeros((n, n)); PU = np.zeros((n, n)); bU = np.zeros((n, 2)); Ug = np.zeros(n)
    assert _ops().orc_mean_ops(My, dt, re, h, _p(MU), _p(PU), _p(bU), _p(Ug)) == 0
    return MU, PU, bU, Ug


def quad_solve(A, B):
    """A^-1 B solved in binary128 and rounded once (the precalculated inverses
    of Sec. 3.2, Listing 3)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    B2 = B.reshape(B.shape[0], -1)
    X = np.zeros_like(B2)
    assert _ops().orc_solve(A.shape[0], _p(A), B2.shape[1], _p(np.ascontiguousarray(B2)), _p(X)) == 0
    return X.reshape(B.shape)


def fundamental(L):
    """2 pi / L, rounded once to double (kx = n 2 pi / Lx, kz = m 2 pi / Lz, Sec. 2)."""
    return _ops().orc_fundamental(float(L))


# Sub-steps of the CN/RK3 scheme (Sec. 3.1): (h, weights of F^0, F^1, F^2)
RK3_SUBSTEPS = ((0.5, (1.0,)), (1.0, (-1.0, 2.0)), (1.0, (1.0 / 6.0, 4.0 / 6.0, 1.0 / 6.0)))


def cn_rk3(x_t, forcing, update):
    """Generic CN/RK3 step (Sec. 3.1): F^i is evaluated on sub-step state i
    (i = 0 is the state at t); sub-step s combines F^0..F^{s-1} with the weights
    above and always restarts from the state at t."""
    Fs = []
    x = x_t
    for s, (h, wts) in enumerate(RK3_SUBSTEPS):
        Fs.append(forcing(x))
        Ft = _combine(wts, Fs)
        x = update(x_t, Ft, h, s)
    return x


def _combine(wts, Fs):
    if isinstance(Fs[0], tuple):
        return tuple(_combine(wts, [F[i] for F in Fs]) for i in range(len(Fs[0])))
    acc = wts[0] * Fs[0]
    for c, F in zip(wts[1:], Fs[1:]):
        acc = acc + c * F
    return acc


class Channel:
    """One group of ensemble members that share a grid, Re and dt (Secs. 2-3;
    the members are the ensemble of Sec. 4.1)."""

    def __init__(self, mx, my, mz, lx, lz, re, dt, flow="couette",
                 u_wall=1.0, bulk_flux=4.0 / 3.0, shared_mean=False, form="advective"):
        """shared_mean: the S3T-type ensemble of Sec. 4.1 (ensemble simulations of
        statistical state dynamics): the members share their streamwise-mean
        (kx = 0) flow, which every sub-step is driven by the kx = 0 part of the
        nonlinear term and by the plane means <uv>, <wv> averaged over the
        members (the perturbation Reynolds stresses averaged over the ensemble).
        The caller gives every member the same kx = 0 part; it then stays
        identical because every member receives the same kx = 0 forcing.
        form: "advective" N = u . grad u (Sec. 3.1), or "rotational" N = omega x u
        (the two differ by grad |u|^2/2, whose curl vanishes: the v, eta forcings
        agree up to the y-aliasing of the collocation derivative; the mean flow is
        forced by d/dy <uv>, <wv> in both)."""
        assert form in ("advective", "rotational")
        self.form = form
        # optional stochastic forcing (oracle.forcing.StochasticForcing), its
        # step counter and the current step's terms
        self.stochastic = None
        self.fstep = 0
        self._noise = None
        self.shared_mean = shared_mean
        self.mx, self.my, self.mz = mx, my, mz
        self.lx, self.lz, self.re, self.dt = lx, lz, re, dt
        self.flow, self.u_wall, self.bulk_flux = flow, u_wall, bulk_flux
        self.Kx, self.Kz = (mx - 1) // 3, (mz - 1) // 3
        self.nyi = my - 2
        self.y, self.D1, self.D2, self.D4c = grid(my)
        self.w = cc_weights(my)
        self.D1i = self.D1[1:-1, 1:-1]
        a1, a3 = fundamental(lx), fundamental(lz)
        self.kx = np.arange(self.Kx + 1) * a1                 # [n]
        self.kz = np.arange(-self.Kz, self.Kz + 1) * a3       # [m + Kz]
        KX = self.kx[None, :]
        KZ = self.kz[:, None]
        self.k2 = KX * KX + KZ * KZ                           # [m, n]
        self.is_mean = np.zeros_like(self.k2, dtype=bool)
        self.is_mean[self.Kz, 0] = True
        self.k2safe = np.where(self.is_mean, 1.0, self.k2)
        # operators per (n, |m|) and per h (Sec. 3.2, Listings 1 and 3)
        pairs_k2 = np.array([[ (n * a1) * (n * a1) + (m * a3) * (m * a3)
                               for n in range(self.Kx + 1)] for m in range(self.Kz + 1)])
        self.ops = {}
        self.mean_ops = {}
        for h in (0.5, 1.0):
            Mv, Pv, Me, Pe = cn_operators(my, pairs_k2.ravel(), dt, re, h)
            sh = (self.Kz + 1, self.Kx + 1, self.nyi, self.nyi)
            absm = np.abs(np.arange(-self.Kz, self.Kz + 1))
            # expand to every (m, n): operators depend on |m| only
            self.ops[h] = tuple(a.reshape(sh)[absm] for a in (Mv, Pv, Me, Pe))
            self.mean_ops[h] = mean_operators(my, dt, re, h)

    # ---------------------------------------------------------- transforms
    def to_physical(self, c):
        """Kept coefficients [..., 2Kz+1, Kx+1] -> real field [..., Mz, Mx]
        (zero-padded inverse transform; the n = 0 column contributes its
        Hermitian part) (Sec. 3.2)."""
        Kx, Kz = self.Kx, self.Kz
        Z = np.zeros(c.shape[:-2] + (self.mz, self.mx // 2 + 1), dtype=np.complex128)
        Z[..., 0:Kz + 1, 0:Kx + 1] = c[..., Kz:, :]
        if Kz > 0:
            Z[..., self.mz - Kz:, 0:Kx + 1] = c[..., :Kz, :]
        return np.fft.irfft2(Z, s=(self.mz, self.mx), norm="forward")

    def to_spectral(self, f):
        """Real field [..., Mz, Mx] -> coefficients of the kept modes (forward
        transform and 2/3-rule truncation, Sec. 3.2)."""
        Kx, Kz = self.Kx, self.Kz
        F = np.fft.rfft2(f, norm="forward")
        out = np.zeros(f.shape[:-2] + (2 * Kz + 1, Kx + 1), dtype=np.complex128)
        out[..., Kz:, :] = F[..., 0:Kz + 1, 0:Kx + 1]
        if Kz > 0:
            out[..., :Kz, :] = F[..., self.mz - Kz:, 0:Kx + 1]
        return out

    # ------------------------------------------------------ velocity field
    def _ydiff(self, D, f):
        """Apply an (My x My) y-operator along axis 1 of f [e, y, m, n]."""
        return np.einsum("ij,ejmn->eimn", D, f)

    def velocity(self, v, eta, U, W):
        """u, v, w and their nine first derivatives on all My nodes (Sec. 3.2):
        returns dict of [e, My, 2Kz+1, Kx+1] spectral arrays."""
        E = v.shape[0]
        sh = (E, self.my, 2 * self.Kz + 1, self.Kx + 1)
        vf = np.zeros(sh, dtype=np.complex128); vf[:, 1:-1] = v
        ef = np.zeros(sh, dtype=np.complex128); ef[:, 1:-1] = eta
        Dv = self._ydiff(self.D1, vf)
        D2v = self._ydiff(self.D2, vf)
        De = self._ydiff(self.D1, ef)
        ikx = 1j * self.kx[None, None, None, :]
        ikz = 1j * self.kz[None, None, :, None]
        k2 = self.k2safe[None, None]
        u = (ikx * Dv - ikz * ef) / k2
        w = (ikz * Dv + ikx * ef) / k2
        uy = (ikx * D2v - ikz * De) / k2
        wy = (ikz * D2v + ikx * De) / k2
        # the (0, 0) mode carries the mean profiles
        u[:, :, self.Kz, 0] = U
        w[:, :, self.Kz, 0] = W
        uy[:, :, self.Kz, 0] = U @ self.D1.T
        wy[:, :, self.Kz, 0] = W @ self.D1.T
        return {
            "u": u, "ux": ikx * u, "uy": uy, "uz": ikz * u,
            "v": vf, "vx": ikx * vf, "vy": Dv, "vz": ikz * vf,
            "w": w, "wx": ikx * w, "wy": wy, "wz": ikz * w,
        }

    # ---------------------------------------------------------- nonlinear
    def nonlinear(self, v, eta, U, W):
        """Advection terms N_i = u . grad u_i (advective form, Sec. 3.1) on the
        interior planes, transformed and truncated, plus the plane means
        <uv>(y), <wv>(y) on all nodes (zero at the walls)."""
        f = self.velocity(v, eta, U, W)
        p = {k: self.to_physical(a[:, 1:-1]) for k, a in f.items()}
        if self.form == "rotational":
            # omega = curl u from the spectral gradients, then N = omega x u
            ox = p["wy"] - p["vz"]
            oy = p["uz"] - p["wx"]
            oz = p["vx"] - p["uy"]
            Nu = oy * p["w"] - oz * p["v"]
            Nv = oz * p["u"] - ox * p["w"]
            Nw = ox * p["v"] - oy * p["u"]
        else:
            Nu = p["u"] * p["ux"] + p["v"] * p["uy"] + p["w"] * p["uz"]
            Nv = p["u"] * p["vx"] + p["v"] * p["vy"] + p["w"] * p["vz"]
            Nw = p["u"] * p["wx"] + p["v"] * p["wy"] + p["w"] * p["wz"]
        E = v.shape[0]
        uv = np.zeros((E, self.my)); wv = np.zeros((E, self.my))
        uv[:, 1:-1] = np.mean(p["u"] * p["v"], axis=(-2, -1))
        wv[:, 1:-1] = np.mean(p["w"] * p["v"], axis=(-2, -1))
        N = [self.to_spectral(Nu), self.to_spectral(Nv), self.to_spectral(Nw)]
        if self.shared_mean:
            # kx = 0 column and plane means: the average over the members
            for a in N:
                a[:, :, :, 0] = np.mean(a[:, :, :, 0], axis=0)[None]
            uv = np.broadcast_to(np.mean(uv, axis=0), uv.shape).copy()
            wv = np.broadcast_to(np.mean(wv, axis=0), wv.shape).copy()
        return N[0], N[1], N[2], uv, wv

    def forcing(self, state):
        """F, G of Eqs. (Dv_F), (eta) and the mean forcings d/dy<uv>, d/dy<wv>
        (Eqs. U00, W00), on the interior nodes."""
        v, eta, U, W = state
        Nu, Nv, Nw, uv, wv = self.nonlinear(v, eta, U, W)
        ikx = 1j * self.kx[None, None, None, :]
        ikz = 1j * self.kz[None, None, :, None]
        phi = ikx * Nu + ikz * Nw
        F = -self.k2[None, None] * Nv - self._yint(self.D1i, phi)
        G = ikz * Nu - ikx * Nw
        F[:, :, self.Kz, 0] = 0.0
        G[:, :, self.Kz, 0] = 0.0
        if self._noise is not None:
            # stochastic forcing of this step, the same in all three sub-steps
            Fn, Gn = self._noise
            F[:, :, :, self.stochastic.n] += Fn
            G[:, :, :, self.stochastic.n] += Gn
        fU = (uv @ self.D1.T)[:, 1:-1]
        fW = (wv @ self.D1.T)[:, 1:-1]
        return (F, G, fU, fW)

    def _yint(self, D, f):
        return np.einsum("ij,ejmn->eimn", D, f)

    # -------------------------------------------------------------- update
    def update(self, state_t, Ft, h, s=None):
        """CN sub-step from the state at t (Eqs. CN1-CN4, Listing 4)."""
        v, eta, U, W = state_t
        F, G, fU, fW = Ft
        Mv, Pv, Me, Pe = self.ops[h]
        vn = np.einsum("mnij,ejmn->eimn", Mv, v) + np.einsum("mnij,ejmn->eimn", Pv, F)
        en = np.einsum("mnij,ejmn->eimn", Me, eta) + np.einsum("mnij,ejmn->eimn", Pe, G)
        vn[:, :, self.Kz, 0] = 0.0
        en[:, :, self.Kz, 0] = 0.0
        MU, PU, bU, Ug = self.mean_ops[h]
        walls_U = U[:, [0, -1]]
        walls_W = W[:, [0, -1]]
        Ui = U[:, 1:-1] @ MU.T + walls_U @ bU.T + fU @ PU.T
        Wi = W[:, 1:-1] @ MU.T + walls_W @ bU.T + fW @ PU.T
        Un = U.copy(); Wn = W.copy()
        gamma = np.zeros(U.shape[0])
        if self.flow == "poiseuille":
            # gamma such that the bulk flux of U equals the prescribed value
            flux0 = Ui @ self.w[1:-1] + walls_U @ self.w[[0, -1]]
            flux1 = Ug @ self.w[1:-1]
            gamma = (self.bulk_flux - flux0) / flux1
            Ui = Ui + gamma[:, None] * Ug[None, :]
        Un[:, 1:-1] = Ui
        Wn[:, 1:-1] = Wi
        self.last_gamma = gamma
        return (vn, en, Un, Wn)

    def step(self, state, nsteps=1):
        """Advance (v, eta, U, W) by nsteps full CN/RK3 steps (Sec. 3.1)."""
        x = tuple(np.array(a) for a in state)
        for _ in range(nsteps):
            if self.stochastic is not None:
                self._noise = self.stochastic.terms(self.fstep, x[0].shape[0])
                self.fstep += 1
            x = cn_rk3(x, self.forcing, self.update)
        self._noise = None
        return x

    # --------------------------------------------------------- statistics
    def stats(self, state):
        """One-point statistics per member (Sec. 4): volume-averaged kinetic
        energy (total and without the mean mode), wall shear dU/dy at both walls,
        bulk flux, max |div u|, the CFL number and profiles U, W, <u'u'>,
        <v'v'>, <w'w'>, <u'v'>."""
        v, eta, U, W = state
        f = self.velocity(v, eta, U, W)
        cn = np.where(np.arange(self.Kx + 1) == 0, 1.0, 2.0)[None, None, None, :]
        pert = ~self.is_mean[None, None]

        def corr(a, b):
            return np.sum(np.real(a * np.conj(b)) * cn * pert, axis=(-2, -1))

        def corr_int(a, b):
            # perturbation correlations on the interior nodes; the no-slip walls
            # carry none (the discrete Dv there is not part of the solution)
            c = corr(a, b)
            c[:, 0] = 0.0
            c[:, -1] = 0.0
            return c

        uu = corr_int(f["u"], f["u"]); vv = corr_int(f["v"], f["v"]); ww = corr_int(f["w"], f["w"])
        uv = corr_int(f["u"], f["v"])
        e_pert = 0.25 * ((uu + vv + ww) @ self.w)
        e_mean = 0.25 * ((U ** 2 + W ** 2) @ self.w)
        dU = U @ self.D1.T
        # dissipation (1/V)(1/Re) int |grad u|^2 dV = (1/(2 Re)) int <|grad u|^2> dy,
        # mean profiles included
        grads = ("ux", "uy", "uz", "vx", "vy", "vz", "wx", "wy", "wz")
        gg = sum(corr(f[k], f[k]) for k in grads) + dU ** 2 + (W @ self.D1.T) ** 2
        dissipation = (gg @ self.w) / (2.0 * self.re)
        # work done by the moving walls (Couette) per unit volume:
        # (1/(2 Re)) [U dU/dy]_{y=-1}^{y=+1}
        wall_work = (U[:, -1] * dU[:, -1] - U[:, 0] * dU[:, 0]) / (2.0 * self.re)
        # CFL number (reading in the module header): velocity on the interior
        # collocation points by the library inverse transform
        yn = self.y
        dy = np.minimum(yn[1:-1] - yn[:-2], yn[2:] - yn[1:-1])
        up, vp, wp = (self.to_physical(f[k][:, 1:-1]) for k in ("u", "v", "w"))   # [e, y, z, x]
        rate = (np.abs(up) * (self.mx / self.lx) + np.abs(vp) / dy[None, :, None, None]
                + np.abs(wp) * (self.mz / self.lz))
        cfl = self.dt * rate.max(axis=(1, 2, 3))
        div = 1j * self.kx[None, None, None, :] * f["u"] + f["vy"] + 1j * self.kz[None, None, :, None] * f["w"]
        div[:, :, self.Kz, 0] = 0.0
        return {
            "e_total": e_pert + e_mean, "e_pert": e_pert,
            "tau_bottom": dU[:, 0], "tau_top": dU[:, -1],
            "bulk_flux": U @ self.w,
            "max_div": np.max(np.abs(div[:, 1:-1]), axis=(1, 2, 3)),
            "dissipation": dissipation, "wall_work": wall_work, "cfl": cfl,
            "U": U, "W": W, "uu": uu, "vv": vv, "ww": ww, "uv": uv,
        }
