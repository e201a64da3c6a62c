// FP64 total energies for reporting (paths, barriers, single points).
//
// The per-step force kernels of the mixed path evaluate per-atom energies in
// FP32; that is enough to order neighbouring images for the upwind tangent
// and to pick the climbing image, but a total over ~1e5 atoms carries errors
// of ~1e-2 eV (in a perfect crystal every atom makes the same rounding
// error).  Reported energies therefore come from these kernels, which redo
// the energy -- and only the energy -- in FP64 from the cell list of the
// configuration being reported: pair vectors from the two-term offsets (exact
// positions), bin displacements and wrap corrections in FP64, then the
// Lennard-Jones, Tersoff or NEP-style energy of Sec. II.B's per-atom split
// summed over atoms in FP64.  Used by cfneb_get_path and cfneb_evaluate, never inside a
// relaxation step.
//
// FP64 arithmetic is scarce on this GPU, so it is spent on the terms only:
// LJ candidates from the cell-list stencil are screened with the leading
// (working-precision) parts first, with a relative margin far above their
// rounding, and only the survivors are formed and tested in FP64; Tersoff
// walks the atom's neighbour list (rebuilt with the cell list) instead of
// the stencil.
#include "common.cuh"

namespace cfneb {

template <typename T>
__device__ inline void pair_vec64(const typename Vec4<T>::type &oi, const typename Vec4<T>::type &oil,
                                  const typename Vec4<T>::type &oj, const typename Vec4<T>::type &ojl,
                                  const double *c, double *r) {
    r[0] = ((double)oj.x + (double)ojl.x) - ((double)oi.x + (double)oil.x) + c[0];
    r[1] = ((double)oj.y + (double)ojl.y) - ((double)oi.y + (double)oil.y) + c[1];
    r[2] = ((double)oj.z + (double)ojl.z) - ((double)oi.z + (double)oil.z) + c[2];
}

// Walk the stencil of slot t and call f(r[3]) for every neighbour entry
// within rc (periodic images included, the atom itself excluded).
template <typename T, typename Fn>
__device__ inline void for_neighbours64(const BandDev &b, int img, int t, const ImgScalars &sc,
                                        double rc2, Fn f) {
    using T4 = typename Vec4<T>::type;
    const size_t base = (size_t)img * b.n;
    const T4 *off = (const T4 *)b.slot_off + base;
    const T4 *offl = (const T4 *)b.slot_off_lo + base;
    const int *start = b.bin_start + (size_t)img * (b.nbins_cap + 1);
    const int nb0 = sc.nb[0], nb1 = sc.nb[1], nb2 = sc.nb[2];
    int b0, b1, b2;
    unpack_bin(b.slot_bin[base + t], b0, b1, b2);
    const T4 oi = off[t], oil = offl[t];
    // leading-part screen: its error (~1e-6 relative in FP32) is far inside
    // the 1e-3 margin; the FP64 test below decides
    const T screen2 = (T)(rc2 * 1.001) + (T)1e-6;
    for (int d0 = -sc.m[0]; d0 <= sc.m[0]; ++d0) {
        int w0 = b0 + d0, t0 = 0;
        while (w0 < 0) { w0 += nb0; --t0; }
        while (w0 >= nb0) { w0 -= nb0; ++t0; }
        for (int d1 = -sc.m[1]; d1 <= sc.m[1]; ++d1) {
            int w1 = b1 + d1, t1 = 0;
            while (w1 < 0) { w1 += nb1; --t1; }
            while (w1 >= nb1) { w1 -= nb1; ++t1; }
            for (int d2 = -sc.m[2]; d2 <= sc.m[2]; ++d2) {
                int w2 = b2 + d2, t2 = 0;
                while (w2 < 0) { w2 += nb2; --t2; }
                while (w2 >= nb2) { w2 -= nb2; ++t2; }
                const int w = (w0 * nb1 + w1) * nb2 + w2;
                double c[3];
                for (int k = 0; k < 3; ++k)
                    c[k] = d0 * sc.bv[k] + d1 * sc.bv[3 + k] + d2 * sc.bv[6 + k] +
                           t0 * sc.dh[k] + t1 * sc.dh[3 + k] + t2 * sc.dh[6 + k];
                const T cx = (T)c[0] - oi.x, cy = (T)c[1] - oi.y, cz = (T)c[2] - oi.z;
                const int q1 = start[w + 1];
                for (int q = start[w]; q < q1; ++q) {
                    const T4 oj = off[q];
                    const T ux = oj.x + cx, uy = oj.y + cy, uz = oj.z + cz;
                    if (!(ux * ux + uy * uy + uz * uz < screen2)) continue;
                    double r[3];
                    pair_vec64<T>(oi, oil, oj, offl[q], c, r);
                    const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
                    if (r2 < rc2 && r2 > 0.0) f(r, r2);
                }
            }
        }
    }
}

// sin a on [0, pi/2] in FP64 by its Taylor series to the a^25 term in
// nested form (truncation below 2e-23 at pi/2); the coefficients
// 1 / ((2k)(2k + 1)) are compile-time constants (an FP64 divide is a long
// dependent sequence on this GPU)
__device__ inline double sin_quarter64(double a) {
    const double a2 = a * a;
    double p = 1.0;
#pragma unroll
    for (int k = 12; k >= 1; --k) p = 1.0 - a2 * (1.0 / (double)((2 * k) * (2 * k + 1))) * p;
    return a * p;
}

// b = (1 + (beta zeta)^n)^(-1/2n) with m2n = -1/2n: x = (beta zeta)^n from
// log and exp; for x < 1e-3 (carbon: x ~ 1e-5) b = exp(m2n log1p(x)) by
// their series (log1p to x^5: 2e-13 relative at the bound, exp to y^6);
// otherwise the library power
__device__ inline double bond_order64(double bz, double n, double m2n) {
    if (!(bz > 0.0)) return 1.0;
    const double x = exp(n * log(bz));
    if (x >= 1e-3) return pow(1.0 + x, m2n);
    const double L = x * (1.0 - x * (0.5 - x * (1.0 / 3.0 - x * (0.25 - x * 0.2))));
    const double y = m2n * L;
    return 1.0 + y * (1.0 + y * (0.5 + y * (1.0 / 6.0 + y * (1.0 / 24.0 + y * (1.0 / 120.0 + y / 720.0)))));
}

// FP64 pair vectors of the neighbour-list entries of slot t within rc
// (periodic images included, the atom itself excluded); returns their count
template <typename T>
__device__ inline int list_vectors64(const BandDev &b, int img, int t, const ImgScalars &sc,
                                     double rc, double *rx, double *ry, double *rz, double *rd) {
    using T4 = typename Vec4<T>::type;
    const size_t base = (size_t)img * b.n;
    const T4 *off = (const T4 *)b.slot_off + base;
    const T4 *offl = (const T4 *)b.slot_off_lo + base;
    const int *nslot = b.nbr_slot + (size_t)img * MAXN_TERSOFF * b.n;
    const int *ncode = b.nbr_code + (size_t)img * MAXN_TERSOFF * b.n;
    const int ne = b.nbr_cnt[base + t];
    int bb[3];
    unpack_bin(b.slot_bin[base + t], bb[0], bb[1], bb[2]);
    const T4 oi = off[t], oil = offl[t];
    int cnt = 0;
    for (int e = 0; e < ne; ++e) {
        const int q = nslot[(size_t)e * b.n + t];
        const int code = ncode[(size_t)e * b.n + t];
        const int dd[3] = {(code & 31) - 16, ((code >> 5) & 31) - 16, ((code >> 10) & 31) - 16};
        int tt[3];
        for (int a = 0; a < 3; ++a) {
            int w = bb[a] + dd[a];
            tt[a] = 0;
            while (w < 0) { w += sc.nb[a]; --tt[a]; }
            while (w >= sc.nb[a]) { w -= sc.nb[a]; ++tt[a]; }
        }
        double c[3];
        for (int k = 0; k < 3; ++k)
            c[k] = dd[0] * sc.bv[k] + dd[1] * sc.bv[3 + k] + dd[2] * sc.bv[6 + k] +
                   tt[0] * sc.dh[k] + tt[1] * sc.dh[3 + k] + tt[2] * sc.dh[6 + k];
        double r[3];
        pair_vec64<T>(oi, oil, off[q], offl[q], c, r);
        const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        if (r2 < rc * rc && r2 > 0.0) {
            rx[cnt] = r[0];
            ry[cnt] = r[1];
            rz[cnt] = r[2];
            rd[cnt] = sqrt(r2);
            ++cnt;
        }
    }
    return cnt;
}

template <typename T>
__global__ void __launch_bounds__(TILE) k_energy64(const Tile *tiles, BandDev *bands) {
    Tile tl = tiles[blockIdx.x];
    BandDev &b = bands[tl.band];
    const ImgScalars &sc = b.sc[tl.img];
    const BandParams *bp = b.bp;
    const int t = tl.t * TILE + threadIdx.x;
    double U = 0.0;
    if (t < b.n) {
        if (bp->kind == 0) {
            const LJParams p = *(const LJParams *)bp->pot;
            const double s2 = p.sigma * p.sigma;
            for_neighbours64<T>(b, tl.img, t, sc, p.rc * p.rc, [&](const double *r, double r2) {
                const double sr6 = s2 * s2 * s2 / (r2 * r2 * r2);
                U += 0.5 * (4.0 * p.eps * (sr6 * sr6 - sr6) - p.ephi_c);
            });
        } else if (bp->kind == 1) {
            const TersoffParams p = *(const TersoffParams *)bp->pot;
            const double rc = p.R + p.D;
            double rx[MAXN_TERSOFF], ry[MAXN_TERSOFF], rz[MAXN_TERSOFF], rd[MAXN_TERSOFF];
            const int cnt = list_vectors64<T>(b, tl.img, t, sc, rc, rx, ry, rz, rd);
            const double pi = 3.14159265358979323846;
            const double c2d2 = p.c * p.c / (p.d * p.d), d2 = p.d * p.d;
            const double pi_4D = 0.25 * pi / p.D, m2n = -0.5 / p.n;
            double fc[MAXN_TERSOFF], ir[MAXN_TERSOFF];
            for (int k = 0; k < cnt; ++k) {
                const double sk = rd[k] - p.R;
                const double sn = sin_quarter64(pi_4D * (p.D - sk));
                fc[k] = sk <= -p.D ? 1.0 : (sk >= p.D ? 0.0 : sn * sn);
                ir[k] = rcp64(rd[k]);
            }
            for (int j = 0; j < cnt; ++j) {
                if (fc[j] == 0.0) continue;  // beyond R + D
                double zeta = 0.0;
                for (int k = 0; k < cnt; ++k) {
                    if (k == j) continue;
                    const double cs = (rx[j] * rx[k] + ry[j] * ry[k] + rz[j] * rz[k]) * ir[j] * ir[k];
                    const double u = p.h - cs;
                    const double g = 1.0 + c2d2 * u * u * rcp64(d2 + u * u);
                    zeta += fc[k] * g;
                }
                U += 0.5 * fc[j] * (p.A * exp(-p.lambda1 * rd[j]) -
                                    bond_order64(p.beta * zeta, p.n, m2n) * p.B * exp(-p.lambda2 * rd[j]));
            }
        } else {
            // NEP-style site energy (descriptors and network as in the force
            // kernel), in FP64 from the list's pair vectors
            const double rc = bp->pot[0];
            double rx[MAXN_TERSOFF], ry[MAXN_TERSOFF], rz[MAXN_TERSOFF], rd[MAXN_TERSOFF];
            const int cnt = list_vectors64<T>(b, tl.img, t, sc, rc, rx, ry, rz, rd);
            const double *w = b.nep_w;
            double qd[NEP_ND], gA[MAXN_TERSOFF][NEP_NA];
            for (int d = 0; d < NEP_ND; ++d) qd[d] = 0.0;
            for (int j = 0; j < cnt; ++j) {
                const double fcj = 0.5 * (1.0 + cospi(rd[j] / rc));
                const double x = 2.0 * (rd[j] / rc - 1.0) * (rd[j] / rc - 1.0) - 1.0;
                double f[NEP_K], t0 = 1.0, t1 = x;
                f[0] = fcj;
                f[1] = 0.5 * (x + 1.0) * fcj;
                for (int k = 2; k < NEP_K; ++k) {
                    const double t2 = 2.0 * x * t1 - t0;
                    f[k] = 0.5 * (t2 + 1.0) * fcj;
                    t0 = t1;
                    t1 = t2;
                }
                for (int m = 0; m < NEP_NR; ++m)
                    for (int k = 0; k < NEP_K; ++k) qd[m] += w[NEP_OCR + m * NEP_K + k] * f[k];
                for (int m = 0; m < NEP_NA; ++m) {
                    gA[j][m] = 0.0;
                    for (int k = 0; k < NEP_K; ++k) gA[j][m] += w[NEP_OCA + m * NEP_K + k] * f[k];
                }
            }
            for (int j = 0; j < cnt; ++j)
                for (int k = 0; k < cnt; ++k) {
                    const double c = (rx[j] * rx[k] + ry[j] * ry[k] + rz[j] * rz[k]) / (rd[j] * rd[k]);
                    const double P[4] = {c, 1.5 * c * c - 0.5, (2.5 * c * c - 1.5) * c,
                                         (4.375 * c * c - 3.75) * c * c + 0.375};
                    for (int m = 0; m < NEP_NA; ++m)
                        for (int l = 0; l < NEP_L; ++l)
                            qd[NEP_NR + m * NEP_L + l] += gA[j][m] * gA[k][m] * (j == k ? 1.0 : P[l]);
                }
            double Ui = -w[NEP_OB1];
            for (int h = 0; h < NEP_H; ++h) {
                double a = -w[NEP_OB0 + h];
                for (int d = 0; d < NEP_ND; ++d) a += w[NEP_OW0 + h * NEP_ND + d] * qd[d];
                Ui += w[NEP_OW1 + h] * tanh(a);
            }
            U += Ui;
        }
    }
    double acc[1] = {U};
    double tot[1];
    block_sum<1>(acc, tot);
    if (threadIdx.x == 0) b.atom_part[((size_t)tl.img * b.atpi + tl.t) * NPART] = tot[0];
}

// one block per image: E64 = sum of the tile energies (+ P Omega)
__global__ void k_energy_finalize(const ImgRef *imgs, BandDev *bands) {
    ImgRef r = imgs[blockIdx.x];
    BandDev &b = bands[r.band];
    const double *part = b.atom_part + (size_t)r.img * b.atpi * NPART;
    double v[1] = {0.0}, s[1];
    for (int t = threadIdx.x; t < b.atpi; t += blockDim.x) v[0] += part[(size_t)t * NPART];
    block_sum_any<1>(v, s);
    if (threadIdx.x == 0) b.sc[r.img].E64 = s[0] + b.bp->pressure * b.sc[r.img].omega;
}

template <typename T>
void launch_energy64(const Tile *tiles, int ntiles, const ImgRef *imgs, int nimg, BandDev *bands,
                     cudaStream_t s) {
    if (ntiles <= 0 || nimg <= 0) return;
    k_energy64<T><<<ntiles, TILE, 0, s>>>(tiles, bands);
    k_energy_finalize<<<nimg, RED_THREADS, 0, s>>>(imgs, bands);
}
template void launch_energy64<float>(const Tile *, int, const ImgRef *, int, BandDev *,
                                     cudaStream_t);
template void launch_energy64<double>(const Tile *, int, const ImgRef *, int, BandDev *,
                                      cudaStream_t);

}  // namespace cfneb
