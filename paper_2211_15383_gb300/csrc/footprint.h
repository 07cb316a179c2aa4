// Device-memory model of one context: the bytes its allocations reach at most for a
// problem shape (lattice levels, terms of the sum, deflation, block width, restart
// length, precision).  Plain C++, host only.  Used by the request server to reserve
// HBM at admission and by the autotuner to keep its candidates inside a budget.
//
// It is an upper estimate: it sums every allocation of the setup, the deflation
// eigensolver and the estimator as if they were live together, although several of
// them never are, then adds 15 % and 32 MB.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstddef>

namespace mg {

struct Shape {
    int L = 0;                       // levels of the hierarchy
    int nterm_levels = 0;            // leading levels that start a term (the rest serve the solver)
    long long sites[8] = {0}, n[8] = {0};
    int d[8] = {0}, nvec[8] = {0};
    int k = 0;                       // smallest triplets of the last term's operator
    int N = 256;                     // right-hand sides per block
    int m = 24;                      // FGMRES restart length
    int precision = 64;              // mg_precision
    int kcycle = 0;                  // K-cycle steps per coarse-grid correction
};

inline size_t footprint_bytes(const Shape& s) {
    const double N = std::max(1, s.N);
    const double m = std::max(1, s.m);
    const bool f64 = s.precision == 64, bf16 = s.precision == 16;
    const double sz = f64 ? 16 : 8;              // bytes of a complex entry of the V-cycle
    const double G = 608, GA = 2432;             // bounds on reduction row groups
    const int L = s.L;
    const int T = s.nterm_levels > 0 ? s.nterm_levels : L;
    const double n0 = (double)s.n[0], nL = (double)s.n[L - 1];
    double nvmax = 1;
    for (int l = 0; l + 1 < L; ++l) nvmax = std::max(nvmax, (double)s.nvec[l]);
    double b = 0;
    b += (double)s.sites[0] * 2 * 24;                                        // links
    for (int l = 0; l < L; ++l) {
        const double st = (double)s.sites[l], d = s.d[l], n = (double)s.n[l];
        b += st * 5 * d * d * (l > 0 ? 24 : 16);                             // D_l (FP64, FP32)
        if (l + 1 < L) {
            const double nv = s.nvec[l];
            b += n * nv * (40 + 16);                                         // P (FP64, FP32), test vectors, raw
            b += st * 5 * d * 2 * nv * 16;                                   // Galerkin product scratch
        }
        if (l > 0 && l + 1 < L) {
            b += st * d * d * (24 + 16) + st * 5 * d * d * 24;               // M^{-1}, D M^{-1}, work
            if (bf16) b += st * d * d * 80;                                  // BF16 operand tiles
        }
        if (l > 0) b += (2.0 * (double)s.n[l - 1] + n) * N * 16;            // FP64 Galerkin apply
        if (l + 1 < L) {
            b += n * N * sz * 3 + 2.0 * (double)s.n[l + 1] * N * sz;         // V-cycle blocks
            if (bf16 && l > 0) b += 3.0 * st * std::ceil(N / 128) * 8192 + n * N * 8;   // BF16 tiles, rhs
            if (bf16 && l == 0) b += 2.0 * n * N * 4;                        // fine-level BF16 r and p
        }
        if (s.kcycle > 0 && l > 0 && l + 1 < L)
            b += (2.0 * s.kcycle + 1) * n * N * sz + G * (s.kcycle + 1) * N * 16;   // K-cycle bases
        if (l > 0) b += n * N * 16;                                          // estimator block of level l
    }
    b += 2.0 * n0 * nvmax * 16;                                              // setup blocks
    b += nL * nL * 44 + nL * N * 136;                                        // dense coarsest inverse, BF16 solve
    b += (2 * m + 1) * n0 * (N * sz + nvmax * 16);                           // FGMRES bases
    b += G * (m + 1) * N * 16 + N * (m + 1) * (m + 4) * 16;                  // Gram-Schmidt partials, Hessenberg
    b += n0 * N * 56;                                                        // refinement blocks
    b += n0 * N * 32;                                                        // noise and solution blocks
    b += G * N * 16 * 6 + GA * N * 8;                                        // reduction partials
    if (s.k > 0) {
        const int ld = T - 1;                                                // the deflated level
        const double nD = (double)s.n[ld], k = s.k;
        const double bb = std::min(nD, std::max(2 * k, k + 16));
        // eigensolver blocks on the deflated level and on the coarser levels that give
        // it its start block (each with room for the block)
        for (int l = ld; l < L; ++l) {
            if (l > ld && (double)s.n[l] < 2 * bb) break;
            b += 5 * (double)s.n[l] * bb * 16;
        }
        // small blocks; partials of the block products (row groups: enough to fill the
        // GPU for FP64, one per 16384 rows for the FP32 form)
        const double tiles = std::ceil(bb / 32) * std::ceil(bb / 32);
        const double groups = std::max(std::ceil(4 * 152 / tiles), std::ceil(nD / 16384));
        b += 5 * bb * bb * 16 + 2 * groups * bb * bb * 16;
        b += 5 * bb * bb * 16;                                               // Jacobi and Cholesky work
        if (bb > N) b += 2 * nD * N * 16;                                    // column chunks of the solves
        b += 2 * nD * k * 16 + G * k * 16;                                   // triplets
        b += 2 * k * N * 16 + G * k * N * 16;                                // FP64 deflation projections
        if (bf16) {
            const double rows = std::ceil(4 * k / 128) * 128, nt = N >= 256 ? 256 : (N > 64 ? 128 : 64);
            const double ncols = std::ceil(N / nt) * nt;
            b += rows * nD * 2 + ncols * nD * 2 + 16 * rows * ncols * 4;     // BF16 factors, packed block, partials
        }
    }
    return (size_t)(b * 1.15) + ((size_t)32 << 20);
}

}  // namespace mg
