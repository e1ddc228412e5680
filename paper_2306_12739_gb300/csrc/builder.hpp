// Host-side operator builder of the channel DNS (double-double, rounded once).
#pragma once
#include <vector>
#include <cstddef>

namespace dnsb {

struct GridOps {
    int my = 0;
    std::vector<double> y;      // [My] ascending nodes
    std::vector<double> D1;     // [My*My]
    std::vector<double> D2;     // [My*My]  = D1 * D1
    std::vector<double> D4c;    // [(My-2)^2] clamped fourth derivative (interior)
    std::vector<double> ccw;    // [My] Clenshaw-Curtis weights
};

// Per sub-step length h: CN operators of every wavenumber pair p = |m|*(Kx+1) + n.
struct CnOps {
    std::vector<double> Mv, Pv, Me, Pe;  // [npairs][Ny][Ny] each, Ny = My - 2
    std::vector<double> MU, PU, bU, Ug;  // mean flow: [Ny][Ny], [Ny][Ny], [Ny][2], [Ny]
    std::vector<double> PD;              // PU * D1[interior rows, all nodes]: [Ny][My]
};

GridOps build_grid(int My);

// k2[p] for every pair p; returns false if a matrix is singular.
bool build_cn(const GridOps& g, const std::vector<double>& k2, double dt, double re, double h,
              CnOps* out, int nthreads);

// 2 pi / L rounded once to double.
double fundamental(double L);

// exp(-2 pi i t / N), t = 0..N-1, interleaved (re, im), rounded once to double.
std::vector<double> twiddles(int N);

}  // namespace dnsb
