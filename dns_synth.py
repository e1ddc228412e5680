"""Seeded synthetic initial states for the ensemble channel DNS.

This module only manufactures inputs: random numbers and the shapes they are
poured into.  It holds none of the time-stepping arithmetic, and both the CPU
oracle (through the tests) and the GPU library (through the binding) consume
what it returns, so the two sides always start from identical bytes.

Random numbers come from a counter-based SplitMix64 stream (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): the k-th draw of
seed s is mix64(s * 0xD1342543DE82EF95 + (k + 1) * 0x9E3779B97F4A7C15) with
SplitMix64's finaliser as mix64, mapped to (0, 1) with 53 bits and to normals by
Box-Muller.

State recipe (the paper gives none; every parameter is an input):
  * nodes y_j = -cos(pi j / (My - 1)), j = 0..My-1 (ascending)
  * mean flow: Couette U = u_wall * y, Poiseuille U = 1 - y^2, W = 0
  * for each kept mode (n, m) != (0, 0) with n <= n_max and |m| <= m_max:
      v_hat(y)   = (1 - y^2)^2 * sum_{p<=4} a_p T_p(y)
      eta_hat(y) = (1 - y^2)   * sum_{p<=4} b_p T_p(y)
    with a_p, b_p complex standard normals times the mode weight
      'flat'      : 1
      'kolmogorov': sqrt((1 + |k| / k1) ** (-5/3 - 1)),  |k| = sqrt(kx^2 + kz^2),
                    k1 = 2 pi / Lx  (a -5/3 shell spectrum, 2-D shell density)
  * the n = 0 column is made Hermitian in m (v_hat(0, -m) = conj v_hat(0, m))
  * each member is rescaled so that
      sqrt( mean_j sum_{modes} c_n (|v_hat_j|^2 + |eta_hat_j|^2) ) = amplitude
    over the interior nodes, with c_0 = 1 and c_n = 2 for n >= 1.

Layout of the returned arrays (also the library's host layout):
  v, eta : complex128 [members][My-2][2 Kz + 1][Kx + 1]  (m index = m + Kz)
  U, W   : float64    [members][My]
with Kx = (Mx - 1) // 3 and Kz = (Mz - 1) // 3.
"""
import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _mix64(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, counters) -> np.ndarray:
    """k-th draws of stream `seed`, uniform on (0, 1)."""
    k = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * np.uint64(0xD1342543DE82EF95)
        z = s + (k + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)
    z = _mix64(z)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed: int, counters) -> np.ndarray:
    """Standard normals by Box-Muller from draws 2k and 2k+1 of stream `seed`."""
    k = np.asarray(counters, dtype=np.uint64)
    u1 = uniform(seed, 2 * k)
    u2 = uniform(seed, 2 * k + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def truncation(M: int) -> int:
    """Largest retained wavenumber index for an M-point periodic grid (2/3 rule)."""
    return (M - 1) // 3


def nodes(My: int) -> np.ndarray:
    y = -np.cos(np.pi * np.arange(My) / (My - 1))
    y[0], y[-1] = -1.0, 1.0
    if (My - 1) % 2 == 0:
        y[(My - 1) // 2] = 0.0
    return y


def make_state(mx, my, mz, lx, lz, flow, members, seed0, amplitude,
               n_max=None, m_max=None, spectrum="flat", u_wall=1.0):
    """Seeded initial ensemble; member e uses seed `seed0 + e`.

    amplitude: scalar or per-member sequence.  n_max / m_max: highest |n|, |m|
    that receive noise (default: every kept mode)."""
    Kx, Kz = truncation(mx), truncation(mz)
    n_max = Kx if n_max is None else min(n_max, Kx)
    m_max = Kz if m_max is None else min(m_max, Kz)
    nyi = my - 2
    y = nodes(my)
    yi = y[1:-1]
    amp = np.broadcast_to(np.asarray(amplitude, dtype=np.float64), (members,))
    # Chebyshev polynomials T_0..T_4 at the interior nodes
    T = np.cos(np.arange(5)[:, None] * np.arccos(np.clip(yi, -1.0, 1.0))[None, :])
    wv = (1.0 - yi ** 2) ** 2
    we = (1.0 - yi ** 2)
    a1 = 2.0 * np.pi / lx
    a3 = 2.0 * np.pi / lz
    v = np.zeros((members, nyi, 2 * Kz + 1, Kx + 1), dtype=np.complex128)
    eta = np.zeros_like(v)
    n_idx, m_idx = np.meshgrid(np.arange(Kx + 1), np.arange(-Kz, Kz + 1), indexing="xy")
    for e in range(members):
        seed = seed0 + e
        # one block of 4 * 5 normals per (m, n) slot: (a re, a im, b re, b im) x p
        cnt = np.arange((2 * Kz + 1) * (Kx + 1) * 20, dtype=np.uint64)
        z = normal(seed, cnt).reshape(2 * Kz + 1, Kx + 1, 4, 5)
        a = z[:, :, 0, :] + 1j * z[:, :, 1, :]
        b = z[:, :, 2, :] + 1j * z[:, :, 3, :]
        kk = np.sqrt((n_idx * a1) ** 2 + (m_idx * a3) ** 2)
        if spectrum == "kolmogorov":
            wgt = np.sqrt((1.0 + kk / a1) ** (-5.0 / 3.0 - 1.0))
        elif spectrum == "flat":
            wgt = np.ones_like(kk)
        else:
            raise ValueError(spectrum)
        mask = (n_idx <= n_max) & (np.abs(m_idx) <= m_max) & ~((n_idx == 0) & (m_idx == 0))
        wgt = np.where(mask, wgt, 0.0)
        ve = np.einsum("mnp,pj->jmn", a * wgt[:, :, None], T) * wv[:, None, None]
        ee = np.einsum("mnp,pj->jmn", b * wgt[:, :, None], T) * we[:, None, None]
        # Hermitian n = 0 column: m < 0 mirrors m > 0
        for arr in (ve, ee):
            arr[:, :Kz, 0] = np.conj(arr[:, :Kz:-1, 0]) if Kz > 0 else arr[:, :Kz, 0]
            arr[:, Kz, 0] = 0.0
        cn = np.where(np.arange(Kx + 1) == 0, 1.0, 2.0)
        ms = (np.sum(cn * (np.abs(ve) ** 2 + np.abs(ee) ** 2)) / nyi)
        scale = amp[e] / np.sqrt(ms) if ms > 0 else 0.0
        v[e] = ve * scale
        eta[e] = ee * scale
    if flow == "couette":
        U = np.tile(u_wall * y, (members, 1))
    elif flow == "poiseuille":
        U = np.tile(1.0 - y ** 2, (members, 1))
    else:
        raise ValueError(flow)
    W = np.zeros((members, my))
    return {"v": v, "eta": eta, "U": U, "W": W}


def make_disturbances(my, mz, lz, members, seed0, amplitude=1.0, m_max=None):
    """Seeded disturbance vectors of one streamwise wavenumber: member e uses
    seed `seed0 + e`; for every kz index |m| <= m_max (default all kept)
      v_hat(y) = (1 - y^2)^2 sum_{p<=4} a_p T_p(y),  eta_hat(y) = (1 - y^2) sum_{p<=4} b_p T_p(y)
    with complex standard normals a_p, b_p (no Hermitian constraint: a single
    kx != 0 column), rescaled like make_state.  Returns complex128
    [members][My-2][2 Kz + 1] arrays v, eta."""
    Kz = truncation(mz)
    m_max = Kz if m_max is None else min(m_max, Kz)
    nyi = my - 2
    yi = nodes(my)[1:-1]
    amp = np.broadcast_to(np.asarray(amplitude, dtype=np.float64), (members,))
    T = np.cos(np.arange(5)[:, None] * np.arccos(np.clip(yi, -1.0, 1.0))[None, :])
    v = np.zeros((members, nyi, 2 * Kz + 1), dtype=np.complex128)
    eta = np.zeros_like(v)
    mask = (np.abs(np.arange(-Kz, Kz + 1)) <= m_max).astype(np.float64)
    for e in range(members):
        cnt = np.arange((2 * Kz + 1) * 20, dtype=np.uint64)
        z = normal(seed0 + e, cnt).reshape(2 * Kz + 1, 4, 5)
        a = (z[:, 0, :] + 1j * z[:, 1, :]) * mask[:, None]
        b = (z[:, 2, :] + 1j * z[:, 3, :]) * mask[:, None]
        ve = np.einsum("mp,pj->jm", a, T) * ((1.0 - yi ** 2) ** 2)[:, None]
        ee = np.einsum("mp,pj->jm", b, T) * (1.0 - yi ** 2)[:, None]
        ms = np.sum(np.abs(ve) ** 2 + np.abs(ee) ** 2) / nyi
        s = amp[e] / np.sqrt(ms) if ms > 0 else 0.0
        v[e] = ve * s
        eta[e] = ee * s
    return {"v": v, "eta": eta}


def make_base_flow(my, mz, lz, flow, seed, streak=0.2, roll=0.02, harmonics=3, u_wall=1.0):
    """Seeded streamwise-mean base flow (U, V, W) on the (My, Mz) grid, walls
    included, y ascending, z_k = k Lz / Mz:
      U = laminar + streak * (1 - y^2) sum_{m=1..H} (c_m cos m b z + s_m sin m b z)
      psi = roll * (1 - y^2)^2 (1 + 0.3 y) sum_{m=1..H} (p_m cos m b z + q_m sin m b z)
      V = d psi / dz,  W = -d psi / dy       (b = 2 pi / Lz)
    so (V, W) is divergence-free and every component vanishes at the walls
    except the laminar U.  Coefficients are standard normals of stream `seed`;
    the y-factors are polynomials (degrees 2, 5 and 4)."""
    y = nodes(my)
    zk = np.arange(mz) * (lz / mz)
    b = 2.0 * np.pi / lz
    z = normal(seed, np.arange(4 * harmonics, dtype=np.uint64)).reshape(4, harmonics)
    c, s, p, q = z
    m = np.arange(1, harmonics + 1)[:, None]
    cz = np.cos(m * b * zk[None, :])
    sz = np.sin(m * b * zk[None, :])
    S_u = (c[:, None] * cz + s[:, None] * sz).sum(0)
    S_psi = (p[:, None] * cz + q[:, None] * sz).sum(0)
    dS_psi = (m * b * (-p[:, None] * sz + q[:, None] * cz)).sum(0)
    lam = u_wall * y if flow == "couette" else 1.0 - y ** 2
    U = lam[:, None] + streak * (1.0 - y ** 2)[:, None] * S_u[None, :]
    g = 1.0 - y ** 2                        # exactly 0 at the walls
    fpsi = g * g * (1.0 + 0.3 * y)
    dfpsi = -4.0 * y * g * (1.0 + 0.3 * y) + 0.3 * g * g
    V = roll * fpsi[:, None] * dS_psi[None, :]
    W = -roll * dfpsi[:, None] * S_psi[None, :]
    return {"U": U, "V": V, "W": W}
