// Host-side operator builder (paper Sec. 2 and Sec. 3.2, Listings 1 and 3).
//
// All arithmetic is double-double (dd.hpp), so the operators are exact to far
// beyond double precision before being rounded once; results are bit-identical
// on x86-64 and aarch64 hosts.
//
//  * nodes y_j = -cos(pi j / (My-1)) (cheb, flipped to ascending y);
//  * D1 from the barycentric formula with the closed-form Gauss-Lobatto weights
//    w_j = (-1)^j delta_j (delta = 1/2 at the ends), diagonal by the
//    negative-sum rule; D2 = D1 D1 (Listing 1);
//  * clamped D4c (cheb4bc, Weideman & Reddy 2000, cited in Sec. 2): fourth
//    derivative of (1-y^2)^2 q(y) with q the interpolant of v_j/(1-y_j^2)^2 on the
//    interior nodes; the interior derivative matrices of q come from Welfert's
//    recursion (SIAM J. Numer. Anal. 34, 1997) and are combined by Leibniz's rule;
//  * per pair and h: A, B of Eq. CN1 multiplied through by Delta (v) and of
//    Eq. CN2 (eta), factorised by LU with partial pivoting, M = A^{-1} B,
//    P = -h dt A^{-1};
//  * mean flow (Eqs. CN3/CN4): wall columns moved to the right-hand side;
//  * Clenshaw-Curtis weights from the closed form of Trefethen's clencurt
//    construction (cosine sums).
#include "builder.hpp"
#include "dd.hpp"

#include <atomic>
#include <thread>

using ddm::dd;

namespace dnsb {

namespace {

// nodes in double-double: y_j = -cos(pi j / N) = sin(pi (2j - N) / (2N))
std::vector<dd> nodes_dd(int My) {
    int N = My - 1;
    std::vector<dd> y(My);
    for (int j = 0; j < My; ++j) {
        dd s, c;
        ddm::sincos_pi_rational(2LL * j - N, 2LL * N, &s, &c);
        y[j] = s;
    }
    y[0] = dd(-1.0);
    y[N] = dd(1.0);
    if (N % 2 == 0) y[N / 2] = dd(0.0);
    return y;
}

using Mat = std::vector<dd>;

Mat matmul(int n, const Mat& A, const Mat& B) {
    Mat C((size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            dd a = A[(size_t)i * n + k];
            if (a.hi == 0.0 && a.lo == 0.0) continue;
            for (int j = 0; j < n; ++j) C[(size_t)i * n + j] += a * B[(size_t)k * n + j];
        }
    return C;
}

// Higher derivative matrices D^(1..4) of the interpolant on arbitrary distinct
// nodes x (n of them), Welfert's recursion:
//   D^(m)_jk = (m / (x_j - x_k)) (c_j/c_k D^(m-1)_jj - D^(m-1)_jk),  j != k,
//   D^(m)_jj = -sum_{k != j} D^(m)_jk,
// with c_j = prod_{i != j} (x_j - x_i).
void welfert(int n, const std::vector<dd>& x, Mat out[4]) {
    std::vector<dd> c(n);
    for (int j = 0; j < n; ++j) {
        dd p(1.0);
        for (int i = 0; i < n; ++i) if (i != j) p = p * (x[j] - x[i]);
        c[j] = p;
    }
    Mat prev((size_t)n * n);
    for (int j = 0; j < n; ++j) prev[(size_t)j * n + j] = dd(1.0);
    for (int m = 1; m <= 4; ++m) {
        Mat cur((size_t)n * n);
        for (int j = 0; j < n; ++j) {
            dd s;
            for (int k = 0; k < n; ++k) {
                if (k == j) continue;
                dd v = dd((double)m) / (x[j] - x[k]) *
                       (c[j] / c[k] * prev[(size_t)j * n + j] - prev[(size_t)j * n + k]);
                cur[(size_t)j * n + k] = v;
                s += v;
            }
            cur[(size_t)j * n + j] = -s;
        }
        out[m - 1] = cur;
        prev = cur;
    }
}

// Solve A X = B in place (A n x n, B n x m) by LU with partial pivoting.
bool lu_solve(int n, Mat& A, int m, Mat& B) {
    std::vector<int> piv(n);
    for (int k = 0; k < n; ++k) {
        int p = k;
        dd best = ddm::ddabs(A[(size_t)k * n + k]);
        for (int i = k + 1; i < n; ++i) {
            dd a = ddm::ddabs(A[(size_t)i * n + k]);
            if (best < a) { best = a; p = i; }
        }
        if (best.hi == 0.0) return false;
        if (p != k) {
            for (int j = 0; j < n; ++j) std::swap(A[(size_t)k * n + j], A[(size_t)p * n + j]);
            for (int j = 0; j < m; ++j) std::swap(B[(size_t)k * m + j], B[(size_t)p * m + j]);
        }
        dd inv = dd(1.0) / A[(size_t)k * n + k];
        for (int i = k + 1; i < n; ++i) {
            dd l = A[(size_t)i * n + k] * inv;
            A[(size_t)i * n + k] = l;
            if (l.hi == 0.0) continue;
            for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= l * A[(size_t)k * n + j];
            for (int j = 0; j < m; ++j) B[(size_t)i * m + j] -= l * B[(size_t)k * m + j];
        }
    }
    // back substitution
    for (int k = n - 1; k >= 0; --k) {
        dd inv = dd(1.0) / A[(size_t)k * n + k];
        for (int j = 0; j < m; ++j) {
            dd s = B[(size_t)k * m + j];
            for (int i = k + 1; i < n; ++i) s -= A[(size_t)k * n + i] * B[(size_t)i * m + j];
            B[(size_t)k * m + j] = s * inv;
        }
    }
    return true;
}

struct GridDD {
    int my;
    std::vector<dd> y;
    Mat D1, D2, D4c;
};

GridDD grid_dd(int My) {
    GridDD g;
    g.my = My;
    g.y = nodes_dd(My);
    int N = My - 1;
    // barycentric weights of the Gauss-Lobatto points: (-1)^j, halved at the ends
    std::vector<double> w(My);
    for (int j = 0; j < My; ++j) w[j] = ((j % 2) ? -1.0 : 1.0) * ((j == 0 || j == N) ? 0.5 : 1.0);
    g.D1.assign((size_t)My * My, dd());
    for (int j = 0; j < My; ++j) {
        dd s;
        for (int k = 0; k < My; ++k) {
            if (k == j) continue;
            dd v = dd(w[k] / w[j]) / (g.y[j] - g.y[k]);
            g.D1[(size_t)j * My + k] = v;
            s += v;
        }
        g.D1[(size_t)j * My + j] = -s;
    }
    g.D2 = matmul(My, g.D1, g.D1);
    // clamped fourth derivative on the interior nodes
    int n = My - 2;
    std::vector<dd> xi(g.y.begin() + 1, g.y.end() - 1);
    Mat T[4];
    welfert(n, xi, T);
    g.D4c.assign((size_t)n * n, dd());
    for (int j = 0; j < n; ++j) {
        dd t = xi[j];
        dd t2 = t * t;
        dd om = (dd(1.0) - t) * (dd(1.0) + t);     // 1 - y^2
        dd w0 = om * om;
        dd w1 = dd(4.0) * t * (t2 - dd(1.0));       // 4y^3 - 4y
        dd w2 = dd(12.0) * t2 - dd(4.0);
        dd w3 = dd(24.0) * t;
        for (int k = 0; k < n; ++k) {
            dd tk = xi[k];
            dd omk = (dd(1.0) - tk) * (dd(1.0) + tk);
            dd wk = omk * omk;
            size_t o = (size_t)j * n + k;
            dd v = w0 * T[3][o] + dd(4.0) * w1 * T[2][o] + dd(6.0) * w2 * T[1][o] + dd(4.0) * w3 * T[0][o];
            if (j == k) v += dd(24.0);
            g.D4c[o] = v / wk;
        }
    }
    return g;
}

// Clenshaw-Curtis weights on x_j = cos(pi j/N) (symmetric, so valid for the
// flipped ordering): w_j = (c_j / N) (1 - sum_{k=1}^{N/2} b_k cos(2 k theta_j) / (4k^2 - 1)),
// c = 1 at the ends and 2 inside, b_k = 1 for k = N/2 (N even), 2 otherwise.
std::vector<double> cc_weights(int My) {
    int N = My - 1;
    std::vector<double> w(My);
    for (int j = 0; j <= N; ++j) {
        dd s(1.0);
        for (int k = 1; k <= N / 2; ++k) {
            double b = (2 * k == N) ? 1.0 : 2.0;
            dd sn, cs;
            ddm::sincos_pi_rational(2LL * k * j, N, &sn, &cs);
            s -= dd(b) * cs / dd((double)(4LL * k * k - 1));
        }
        double c = (j == 0 || j == N) ? 1.0 : 2.0;
        w[j] = (double)(dd(c) * s / dd((double)N));
    }
    return w;
}

std::vector<double> round_all(const Mat& a) {
    std::vector<double> r(a.size());
    for (size_t i = 0; i < a.size(); ++i) r[i] = (double)a[i];
    return r;
}

}  // namespace

GridOps build_grid(int My) {
    GridDD g = grid_dd(My);
    GridOps o;
    o.my = My;
    o.y.resize(My);
    for (int j = 0; j < My; ++j) o.y[j] = (double)g.y[j];
    o.D1 = round_all(g.D1);
    o.D2 = round_all(g.D2);
    o.D4c = round_all(g.D4c);
    o.ccw = cc_weights(My);
    return o;
}

bool build_cn(const GridOps& go, const std::vector<double>& k2, double dt, double re, double h,
              CnOps* out, int nthreads) {
    const int My = go.my;
    GridDD g = grid_dd(My);
    const int n = My - 2;
    const size_t nn = (size_t)n * n;
    Mat D2i(nn);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) D2i[(size_t)i * n + j] = g.D2[(size_t)(i + 1) * My + (j + 1)];
    const dd gg = dd(h) * dd(dt) / (dd(2.0) * dd(re));
    const dd hdt = dd(h) * dd(dt);
    const int np = (int)k2.size();
    out->Mv.assign(np * nn, 0.0); out->Pv.assign(np * nn, 0.0);
    out->Me.assign(np * nn, 0.0); out->Pe.assign(np * nn, 0.0);
    std::atomic<int> next(0), bad(0);
    auto work = [&]() {
        Mat A(nn), B((size_t)n * 2 * n);
        for (;;) {
            int p = next.fetch_add(1);
            if (p >= np) break;
            dd kk(k2[p]);
            // v: A = Delta - g DD, B = [Delta + g DD | -h dt I]
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) {
                    size_t o = (size_t)i * n + j;
                    dd del = D2i[o];
                    dd dd4 = g.D4c[o] - dd(2.0) * kk * D2i[o];
                    if (i == j) { del -= kk; dd4 += kk * kk; }
                    A[o] = del - gg * dd4;
                    B[(size_t)i * 2 * n + j] = del + gg * dd4;
                    B[(size_t)i * 2 * n + n + j] = (i == j) ? -hdt : dd();
                }
            if (!lu_solve(n, A, 2 * n, B)) { bad = 1; continue; }
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) {
                    out->Mv[p * nn + (size_t)i * n + j] = (double)B[(size_t)i * 2 * n + j];
                    out->Pv[p * nn + (size_t)i * n + j] = (double)B[(size_t)i * 2 * n + n + j];
                }
            // eta: A = I - g Delta, B = [I + g Delta | -h dt I]
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) {
                    size_t o = (size_t)i * n + j;
                    dd del = D2i[o];
                    if (i == j) del -= kk;
                    dd id = (i == j) ? dd(1.0) : dd();
                    A[o] = id - gg * del;
                    B[(size_t)i * 2 * n + j] = id + gg * del;
                    B[(size_t)i * 2 * n + n + j] = (i == j) ? -hdt : dd();
                }
            if (!lu_solve(n, A, 2 * n, B)) { bad = 1; continue; }
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) {
                    out->Me[p * nn + (size_t)i * n + j] = (double)B[(size_t)i * 2 * n + j];
                    out->Pe[p * nn + (size_t)i * n + j] = (double)B[(size_t)i * 2 * n + n + j];
                }
        }
    };
    int nt = nthreads > 0 ? nthreads : 1;
    if (nt > np) nt = np > 0 ? np : 1;
    std::vector<std::thread> th;
    for (int t = 1; t < nt; ++t) th.emplace_back(work);
    work();
    for (auto& t : th) t.join();
    if (bad) return false;

    // mean flow, Eqs. CN3/CN4 with the wall columns on the right-hand side:
    // A = I - g D2_int, RHS = [I + g D2_int | -h dt I | 2 g D2[int, 0] | 2 g D2[int, My-1] | h dt 1]
    {
        int m = 2 * n + 3;
        Mat A(nn), B((size_t)n * m);
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j) {
                size_t o = (size_t)i * n + j;
                dd id = (i == j) ? dd(1.0) : dd();
                A[o] = id - gg * D2i[o];
                B[(size_t)i * m + j] = id + gg * D2i[o];
                B[(size_t)i * m + n + j] = (i == j) ? -hdt : dd();
            }
            B[(size_t)i * m + 2 * n] = dd(2.0) * gg * g.D2[(size_t)(i + 1) * My + 0];
            B[(size_t)i * m + 2 * n + 1] = dd(2.0) * gg * g.D2[(size_t)(i + 1) * My + (My - 1)];
            B[(size_t)i * m + 2 * n + 2] = hdt;
        }
        if (!lu_solve(n, A, m, B)) return false;
        out->MU.assign(nn, 0.0); out->PU.assign(nn, 0.0);
        out->bU.assign((size_t)n * 2, 0.0); out->Ug.assign(n, 0.0);
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j) {
                out->MU[(size_t)i * n + j] = (double)B[(size_t)i * m + j];
                out->PU[(size_t)i * n + j] = (double)B[(size_t)i * m + n + j];
            }
            out->bU[(size_t)i * 2 + 0] = (double)B[(size_t)i * m + 2 * n];
            out->bU[(size_t)i * 2 + 1] = (double)B[(size_t)i * m + 2 * n + 1];
            out->Ug[i] = (double)B[(size_t)i * m + 2 * n + 2];
        }
        // PD = PU D1[1..My-2, :]: the mean forcing d/dy <uv> folded into the solve,
        // so that PU (D1 uv) = PD uv (uv vanishes on the walls)
        out->PD.assign((size_t)n * My, 0.0);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < My; ++j) {
                dd acc;
                for (int k = 0; k < n; ++k) acc += B[(size_t)i * m + n + k] * g.D1[(size_t)(k + 1) * My + j];
                out->PD[(size_t)i * My + j] = (double)acc;
            }
    }
    return true;
}

double fundamental(double L) {
    return (double)(dd(2.0) * ddm::dd_pi() / dd(L));
}

std::vector<double> twiddles(int N) {
    std::vector<double> t(2 * (size_t)N);
    for (int k = 0; k < N; ++k) {
        dd s, c;
        ddm::sincos_pi_rational(2LL * k, N, &s, &c);   // angle 2 pi k / N
        t[2 * k] = (double)c;
        t[2 * k + 1] = -(double)s;
    }
    return t;
}

}  // namespace dnsb
