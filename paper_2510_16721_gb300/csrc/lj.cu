// Lennard-Jones energy, forces and virial over the cell list.
//
// phi(r) = 4 eps [(sigma/r)^12 - (sigma/r)^6] - phi(rc) (energy shifted when
// requested); U_i = 1/2 sum_j phi(r_ij) (the per-atom split of Sec. II.B,
// Eq. U).  For a pair potential the force on i due to j of the
// derivation of Eq. V2, f^ij = dU_i/dr^ij - dU_j/dr^ji, is phi'(r) r^ij / r,
// so F_i = sum_j phi'(r) r^ij / r and V = -1/2 sum_ij r^ij (x) f^ij.
//
// One thread per atom, atoms taken in cell-list slot order (neighbouring
// threads share neighbour bins, so their loads hit L1).  Full neighbour
// enumeration (every pair visited from both ends): no atomics, fixed
// summation order.  Arithmetic in T (float on the mixed path) with T
// per-atom accumulators; tile energies and virials are summed in FP64.  The
// epilogue applies the cell filter's atom-row transform F D^T (Sec. II.C).
#include "common.cuh"

namespace cfneb {

template <typename T>
__device__ inline T rcp(T x);
template <>
__device__ inline float rcp<float>(float x) { return __frcp_rn(x); }
template <>
__device__ inline double rcp<double>(double x) { return 1.0 / x; }

template <typename T>
__global__ void __launch_bounds__(TILE) k_lj(const Tile *tiles, BandDev *bands) {
    using T4 = typename Vec4<T>::type;
    Tile tl = tiles[blockIdx.x];
    BandDev &b = bands[tl.band];
    const ImgScalars &sc = b.sc[tl.img];
    const LJParams p = *(const LJParams *)b.bp->pot;
    __shared__ T s_bv[9], s_dh[9], s_D[9];
    __shared__ int s_nb[3], s_m[3];
    if (threadIdx.x < 9) {
        s_bv[threadIdx.x] = (T)sc.bv[threadIdx.x];
        s_dh[threadIdx.x] = (T)sc.dh[threadIdx.x];
        s_D[threadIdx.x] = (T)sc.D[threadIdx.x];
    }
    if (threadIdx.x < 3) {
        s_nb[threadIdx.x] = sc.nb[threadIdx.x];
        s_m[threadIdx.x] = sc.m[threadIdx.x];
    }
    __syncthreads();
    const int n = b.n;
    const int t = tl.t * TILE + threadIdx.x;
    const size_t base = (size_t)tl.img * n;
    const T4 *off = (const T4 *)b.slot_off + base;
    const int *start = b.bin_start + (size_t)tl.img * (b.nbins_cap + 1);
    const T rc2 = (T)(p.rc * p.rc), sig2 = (T)(p.sigma * p.sigma);
    const T rc2_screen = rc2 * (T)1.00001;  // cheap test first, exact test after
    const T eps4 = (T)(4.0 * p.eps), eps24 = (T)(24.0 * p.eps);
    T fx = 0, fy = 0, fz = 0, e = 0;
    T v00 = 0, v01 = 0, v02 = 0, v11 = 0, v12 = 0, v22 = 0;
    int cnt = 0;
    if (t < n) {
        const int bin = b.slot_bin[base + t];
        const int nb1 = s_nb[1], nb2 = s_nb[2];
        const int b0 = bin / (nb1 * nb2), b1 = (bin / nb2) % nb1, b2 = bin % nb2;
        const T4 oi = off[t];
        for (int d0 = -s_m[0]; d0 <= s_m[0]; ++d0) {
            int w0 = b0 + d0, t0 = 0;
            while (w0 < 0) { w0 += s_nb[0]; --t0; }
            while (w0 >= s_nb[0]) { w0 -= s_nb[0]; ++t0; }
            for (int d1 = -s_m[1]; d1 <= s_m[1]; ++d1) {
                int w1 = b1 + d1, t1 = 0;
                while (w1 < 0) { w1 += nb1; --t1; }
                while (w1 >= nb1) { w1 -= nb1; ++t1; }
                for (int d2 = -s_m[2]; d2 <= s_m[2]; ++d2) {
                    int w2 = b2 + d2, t2 = 0;
                    while (w2 < 0) { w2 += nb2; --t2; }
                    while (w2 >= nb2) { w2 -= nb2; ++t2; }
                    const int w = (w0 * nb1 + w1) * nb2 + w2;
                    // displacement between the two bin centres (exact in T
                    // for |delta| <= 1 in orthorhombic cells)
                    const T cx = (d0 * s_bv[0] + d1 * s_bv[3] + d2 * s_bv[6]) +
                                 (t0 * s_dh[0] + t1 * s_dh[3] + t2 * s_dh[6]);
                    const T cy = (d0 * s_bv[1] + d1 * s_bv[4] + d2 * s_bv[7]) +
                                 (t0 * s_dh[1] + t1 * s_dh[4] + t2 * s_dh[7]);
                    const T cz = (d0 * s_bv[2] + d1 * s_bv[5] + d2 * s_bv[8]) +
                                 (t0 * s_dh[2] + t1 * s_dh[5] + t2 * s_dh[8]);
                    const T sx = cx - oi.x, sy = cy - oi.y, sz = cz - oi.z;
                    const int q1 = start[w + 1];
                    for (int q = start[w]; q < q1; ++q) {
                        const T4 oj = off[q];
                        const T ux = oj.x + sx, uy = oj.y + sy, uz = oj.z + sz;
                        if (ux * ux + uy * uy + uz * uz >= rc2_screen) continue;
                        // accepted: pair vector with the small offsets
                        // subtracted first
                        const T rx = (oj.x - oi.x) + cx, ry = (oj.y - oi.y) + cy,
                                rz = (oj.z - oi.z) + cz;
                        const T r2 = rx * rx + ry * ry + rz * rz;
                        // r2 == 0 only for the atom itself at zero shift
                        if (r2 < rc2 && r2 > (T)0) {
                            const T ir2 = rcp<T>(r2);
                            const T sr2 = sig2 * ir2;
                            const T sr6 = sr2 * sr2 * sr2;
                            // phi'(r)/r = 24 eps (sr6 - 2 sr6^2) / r^2
                            const T fr = eps24 * sr6 * ((T)1 - (T)2 * sr6) * ir2;
                            fx += fr * rx;
                            fy += fr * ry;
                            fz += fr * rz;
                            e += sr6 * (sr6 - (T)1);
                            v00 += fr * rx * rx;
                            v01 += fr * rx * ry;
                            v02 += fr * rx * rz;
                            v11 += fr * ry * ry;
                            v12 += fr * ry * rz;
                            v22 += fr * rz * rz;
                            ++cnt;
                        }
                    }
                }
            }
        }
        // generalised atom force F D^T (row vector times D^T)
        T g0 = fx * s_D[0] + fy * s_D[1] + fz * s_D[2];
        T g1 = fx * s_D[3] + fy * s_D[4] + fz * s_D[5];
        T g2 = fx * s_D[6] + fy * s_D[7] + fz * s_D[8];
        const int atom = b.slot_atom[base + t];
        T *F = (T *)b.F + ((size_t)tl.img * b.rows + atom) * 3;
        F[0] = g0;
        F[1] = g1;
        F[2] = g2;
    }
    // U_i = 1/2 sum_j [4 eps (sr12 - sr6) - phi(rc)];  V = -1/2 sum r (x) f
    T acc[8];
    acc[0] = (T)0.5 * (eps4 * e - (T)p.ephi_c * (T)cnt);
    acc[1] = (T)(-0.5) * v00;
    acc[2] = (T)(-0.5) * v01;
    acc[3] = (T)(-0.5) * v02;
    acc[4] = (T)(-0.5) * v11;
    acc[5] = (T)(-0.5) * v12;
    acc[6] = (T)(-0.5) * v22;
    acc[7] = (T)cnt;
    double r8[8];
    block_sum_t<8, T>(acc, r8);
    // symmetric virial, row-major
    const double tot[11] = {r8[0], r8[1], r8[2], r8[3], r8[2], r8[4], r8[5],
                            r8[3], r8[5], r8[6], r8[7]};
    if (threadIdx.x == 0) {
        double *part = b.atom_part + ((size_t)tl.img * b.atpi + tl.t) * NPART;
        for (int k = 0; k < 11; ++k) part[k] = tot[k];
        part[11] = 0.0;
    }
}

template <typename T>
void launch_lj(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s) {
    if (ntiles <= 0) return;
    k_lj<T><<<ntiles, TILE, 0, s>>>(tiles, bands);
}
template void launch_lj<float>(const Tile *, int, BandDev *, cudaStream_t);
template void launch_lj<double>(const Tile *, int, BandDev *, cudaStream_t);

}  // namespace cfneb
