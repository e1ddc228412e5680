// Column tiles of the register-tiled kernels of the mixed path (k_gemm_f32.cu,
// k_step_eo.cu): QT consecutive modes x EBT consecutive members per CTA; the
// work items of their implicit apply.
#pragma once
#include "dns_internal.hpp"

namespace dnsk {
namespace gt {

// Column tile: QT consecutive modes x EBT consecutive members (complex columns).
struct Tile {
    int QT, EBT, NC;   // NC = QT * EBT complex columns
};

// Up to 64 complex columns per tile (32 for tall operators), halved down to 16
// while the grid would hold fewer than three CTAs per SM (152 SMs): first fewer
// modes per tile, then, for large member counts with few modes (linear groups),
// shorter member runs (never below 16 members: 128-byte runs of the H layout).
__host__ __device__ inline Tile tile_of(int E, int ny, int nm, int cap0 = 0) {
    int cap = cap0 > 0 ? cap0 : (ny <= 96 ? 64 : 32);
    Tile t;
    for (;;) {
        t.EBT = E < cap ? E : cap;
        t.QT = cap / t.EBT;
        if (t.QT < 1) t.QT = 1;
        t.NC = t.QT * t.EBT;
        const long long ctas = (long long)((nm + t.QT - 1) / t.QT) * ((E + t.EBT - 1) / t.EBT);
        if (cap <= 16 || ctas >= 3 * 152) break;
        cap /= 2;
    }
    return t;
}

// One work item of the implicit apply: wavenumber pair p, field f (0 v, 1 eta),
// member chunk ch.
struct HelmItem {
    int p, f, e0, ec, nq, q1, q2, NC;
};

__device__ __forceinline__ HelmItem helm_item(const GroupView& g, int p, int f, int ch) {
    HelmItem it;
    const int NKX = g.nkx, n = p % NKX, am = p / NKX;
    const int EC = helm_member_chunk(g);
    it.p = p;
    it.f = f;
    it.e0 = ch * EC;
    it.ec = min(EC, g.E - it.e0);
    it.nq = am > 0 ? 2 : 1;
    it.q1 = (g.kz + am) * NKX + n;
    it.q2 = (g.kz - am) * NKX + n;
    it.NC = it.nq * 2 * it.ec;
    return it;
}

}  // namespace gt
}  // namespace dnsk
