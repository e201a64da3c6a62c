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

// Per-thread LJ accumulators: force on atom i, energy sum, virial, pair count
template <typename T>
struct LJAcc {
    T fx = 0, fy = 0, fz = 0, e = 0;
    T v00 = 0, v01 = 0, v02 = 0, v11 = 0, v12 = 0, v22 = 0;
    int cnt = 0;
    __device__ inline void pair(T rx, T ry, T rz, T sig2, T eps24) {
        const T r2 = rx * rx + ry * ry + rz * rz;
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
};

// One thread per atom in slot order.  The stencil is walked as rows along
// the innermost bin axis: where the row does not wrap around the cell its
// bins are consecutive in the cell list, so the row is one contiguous range
// of atoms (one pair of bin-start loads instead of one per bin) and each
// atom's displacement comes from its own innermost bin index, stored in the
// offset's fourth lane.  Rows that wrap are walked bin by bin.
template <typename T>
__global__ void __launch_bounds__(TILE, sizeof(T) == 4 ? 8 : 4) k_lj(const Tile *tiles, BandDev *bands) {
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
    const T eps4 = (T)(4.0 * p.eps), eps24 = (T)(24.0 * p.eps);
    LJAcc<T> A;
    if (t < n) {
        const int nb0 = s_nb[0], nb1 = s_nb[1], nb2 = s_nb[2];
        const int m2 = s_m[2];
        const T4 oi = off[t];
        const int b2 = (int)oi.w;
        const int bin = b.slot_bin[base + t];
        const int b0 = bin / (nb1 * nb2), b1 = (bin / nb2) % nb1;
        const bool row_ok = (b2 - m2 >= 0) && (b2 + m2 < nb2);
        for (int d0 = -s_m[0]; d0 <= s_m[0]; ++d0) {
            int w0 = b0 + d0, t0 = 0;
            while (w0 < 0) { w0 += nb0; --t0; }
            while (w0 >= nb0) { w0 -= nb0; ++t0; }
            for (int d1 = -s_m[1]; d1 <= s_m[1]; ++d1) {
                int w1 = b1 + d1, t1 = 0;
                while (w1 < 0) { w1 += nb1; --t1; }
                while (w1 >= nb1) { w1 -= nb1; ++t1; }
                const int rowbase = (w0 * nb1 + w1) * nb2;
                // displacement for d2 = 0 (row base) and the wrap remainder
                const T cx = (d0 * s_bv[0] + d1 * s_bv[3]) + (t0 * s_dh[0] + t1 * s_dh[3]);
                const T cy = (d0 * s_bv[1] + d1 * s_bv[4]) + (t0 * s_dh[1] + t1 * s_dh[4]);
                const T cz = (d0 * s_bv[2] + d1 * s_bv[5]) + (t0 * s_dh[2] + t1 * s_dh[5]);
                if (row_ok) {
                    const int q0 = start[rowbase + b2 - m2], q1 = start[rowbase + b2 + m2 + 1];
                    for (int q = q0; q < q1; ++q) {
                        const T4 oj = off[q];
                        const T d2 = oj.w - (T)b2;
                        const T ex = cx + d2 * s_bv[6], ey = cy + d2 * s_bv[7],
                                ez = cz + d2 * s_bv[8];
                        const T ux = (oj.x - oi.x) + ex, uy = (oj.y - oi.y) + ey,
                                uz = (oj.z - oi.z) + ez;
                        const T r2 = ux * ux + uy * uy + uz * uz;
                        // r2 == 0 only for the atom itself at zero shift
                        if (r2 < rc2 && r2 > (T)0) A.pair(ux, uy, uz, sig2, eps24);
                    }
                } else {
                    for (int d2 = -m2; d2 <= m2; ++d2) {
                        int w2 = b2 + d2, t2 = 0;
                        while (w2 < 0) { w2 += nb2; --t2; }
                        while (w2 >= nb2) { w2 -= nb2; ++t2; }
                        const T ex = cx + (d2 * s_bv[6] + t2 * s_dh[6]);
                        const T ey = cy + (d2 * s_bv[7] + t2 * s_dh[7]);
                        const T ez = cz + (d2 * s_bv[8] + t2 * s_dh[8]);
                        const int q1 = start[rowbase + w2 + 1];
                        for (int q = start[rowbase + w2]; q < q1; ++q) {
                            const T4 oj = off[q];
                            const T ux = (oj.x - oi.x) + ex, uy = (oj.y - oi.y) + ey,
                                    uz = (oj.z - oi.z) + ez;
                            const T r2 = ux * ux + uy * uy + uz * uz;
                            if (r2 < rc2 && r2 > (T)0) A.pair(ux, uy, uz, sig2, eps24);
                        }
                    }
                }
            }
        }
        // generalised atom force F D^T (row vector times D^T)
        const T g0 = A.fx * s_D[0] + A.fy * s_D[1] + A.fz * s_D[2];
        const T g1 = A.fx * s_D[3] + A.fy * s_D[4] + A.fz * s_D[5];
        const T g2 = A.fx * s_D[6] + A.fy * s_D[7] + A.fz * s_D[8];
        const int atom = b.slot_atom[base + t];
        T *F = (T *)b.F + ((size_t)tl.img * b.rows + atom) * 3;
        F[0] = g0;
        F[1] = g1;
        F[2] = g2;
    }
    // U_i = 1/2 sum_j [4 eps (sr12 - sr6) - phi(rc)];  V = -1/2 sum r (x) f
    T acc[8];
    acc[0] = (T)0.5 * (eps4 * A.e - (T)p.ephi_c * (T)A.cnt);
    acc[1] = (T)(-0.5) * A.v00;
    acc[2] = (T)(-0.5) * A.v01;
    acc[3] = (T)(-0.5) * A.v02;
    acc[4] = (T)(-0.5) * A.v11;
    acc[5] = (T)(-0.5) * A.v12;
    acc[6] = (T)(-0.5) * A.v22;
    acc[7] = (T)A.cnt;
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
