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

// sigma^2 / r^2: FP32 by the fast division intrinsic (2 ulp: ~1e-6 of a
// pair force, far inside the mixed path's 1e-4 force tolerance), FP64 exact
__device__ inline float lj_sr2(float sig2, float r2) { return __fdividef(sig2, r2); }
__device__ inline double lj_sr2(double sig2, double r2) { return sig2 / r2; }

// Per-thread LJ accumulators: force on atom i, energy sum, virial, pair count
template <typename T>
struct LJAcc {
    T fx = 0, fy = 0, fz = 0, e = 0;
    T v00 = 0, v01 = 0, v02 = 0, v11 = 0, v12 = 0, v22 = 0;
    int cnt = 0;
    // pair vector (rx, ry, rz) with |r|^2 = r2; c24 = 24 eps / sigma^2
    __device__ inline void pair(T rx, T ry, T rz, T r2, T sig2, T c24) {
        const T sr2 = lj_sr2(sig2, r2);
        const T sr6 = sr2 * sr2 * sr2;
        // phi'(r)/r = 24 eps (sr6 - 2 sr6^2) / r^2
        const T fr = c24 * sr2 * sr6 * ((T)1 - (T)2 * sr6);
        const T frx = fr * rx, fry = fr * ry, frz = fr * rz;
        fx += frx;
        fy += fry;
        fz += frz;
        e += sr6 * (sr6 - (T)1);
        v00 += frx * rx;
        v01 += frx * ry;
        v02 += frx * rz;
        v11 += fry * ry;
        v12 += fry * rz;
        v22 += frz * rz;
        ++cnt;
    }
};

// floor(a / b) for b > 0
__device__ inline int floor_div(int a, int b) { return a >= 0 ? a / b : -((b - 1 - a) / b); }

// Code of a (bin offset d, periodic wrap t) combination along one axis.  For
// any bin of an axis of nb bins, t is floor(d / nb) or floor(d / nb) + 1, so
// 2 (d + m) + (t - floor(d / nb)) < 2 (2m + 1) <= 30 identifies it.
__device__ inline int axis_code(int d, int t, int m, int nb) {
    return 2 * (d + m) + (t - floor_div(d, nb));
}

// Neighbour-list entry: slot in bits 0-16, i0 + LJ_AXIS i1 in bits 17-26 and
// i2 in bits 27-31 (i_a the axis codes).  The list path therefore needs
// n <= 2^17 atoms per image.
constexpr int LJ_AXIS = 30;
// entries the list force kernel takes per iteration (lists are padded to it)
constexpr int LJ_UNROLL = 4;
__device__ inline uint32_t lj_entry(int q, int i01, int i2) {
    return (uint32_t)q | ((uint32_t)i01 << 17) | ((uint32_t)i2 << 27);
}

// Visits every cell-list candidate of the atom with offset oi in bin `bin`:
// visit(q, ux, uy, uz, i01, i2) with (ux, uy, uz) the pair vector to slot q
// and i01 = i0 + LJ_AXIS i1, i2 the axis codes of its (offset, wrap).
// The stencil is walked as rows along the innermost bin axis: where the row
// does not wrap around the cell its bins are consecutive in the cell list,
// so the row is one contiguous range of atoms (one pair of bin-start loads
// instead of one per bin) and each atom's displacement comes from its own
// innermost bin index, stored in the offset's fourth lane.  Rows that wrap
// are walked bin by bin.
template <typename T, typename Visit>
__device__ inline void lj_walk(const typename Vec4<T>::type *off, const int *start,
                               const typename Vec4<T>::type &oi, int bin, const T *s_bv,
                               const T *s_dh, const int *s_nb, const int *s_m, Visit &&visit) {
    using T4 = typename Vec4<T>::type;
    const int nb0 = s_nb[0], nb1 = s_nb[1], nb2 = s_nb[2];
    const int m0 = s_m[0], m1 = s_m[1], m2 = s_m[2];
    int b0, b1, b2;
    unpack_bin(bin, b0, b1, b2);
    const bool row_ok = (b2 - m2 >= 0) && (b2 + m2 < nb2);
    for (int d0 = -m0; d0 <= m0; ++d0) {
        int w0 = b0 + d0, t0 = 0;
        while (w0 < 0) { w0 += nb0; --t0; }
        while (w0 >= nb0) { w0 -= nb0; ++t0; }
        const int i0 = axis_code(d0, t0, m0, nb0);
        for (int d1 = -m1; d1 <= m1; ++d1) {
            int w1 = b1 + d1, t1 = 0;
            while (w1 < 0) { w1 += nb1; --t1; }
            while (w1 >= nb1) { w1 -= nb1; ++t1; }
            const int i01 = i0 + LJ_AXIS * axis_code(d1, t1, m1, nb1);
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
                    // no wrap along the row: t2 = 0, and |d2| <= m2 < nb2
                    const int id2 = (int)d2;
                    visit(q, (oj.x - oi.x) + ex, (oj.y - oi.y) + ey, (oj.z - oi.z) + ez, i01,
                          2 * (id2 + m2) + (id2 < 0 ? 1 : 0));
                }
            } else {
                for (int d2 = -m2; d2 <= m2; ++d2) {
                    int w2 = b2 + d2, t2 = 0;
                    while (w2 < 0) { w2 += nb2; --t2; }
                    while (w2 >= nb2) { w2 -= nb2; ++t2; }
                    const int i2 = axis_code(d2, t2, m2, nb2);
                    const T ex = cx + (d2 * s_bv[6] + t2 * s_dh[6]);
                    const T ey = cy + (d2 * s_bv[7] + t2 * s_dh[7]);
                    const T ez = cz + (d2 * s_bv[8] + t2 * s_dh[8]);
                    const int q1 = start[rowbase + w2 + 1];
                    for (int q = start[rowbase + w2]; q < q1; ++q) {
                        const T4 oj = off[q];
                        visit(q, (oj.x - oi.x) + ex, (oj.y - oi.y) + ey, (oj.z - oi.z) + ez,
                              i01, i2);
                    }
                }
            }
        }
    }
}

// Per-block staging of an image's bin geometry and the LJ constants in T
template <typename T>
struct LJGeom {
    T bv[9], dh[9], D[9];
    T rc2, sig2, c24, e4, ephi;   // rc^2, sigma^2, 24 eps / sigma^2, 4 eps, phi(rc)
    T screen;                     // list screen: rl^2 with a 1e-5 relative margin
    int nb[3], m[3];
};
template <typename T>
__device__ inline void lj_stage(LJGeom<T> &g, const ImgScalars &sc, const BandParams &bp) {
    if (threadIdx.x == 0) {
        const LJParams p = *(const LJParams *)bp.pot;
        g.rc2 = (T)(p.rc * p.rc);
        g.sig2 = (T)(p.sigma * p.sigma);
        g.c24 = (T)(24.0 * p.eps / (p.sigma * p.sigma));
        g.e4 = (T)(4.0 * p.eps);
        g.ephi = (T)p.ephi_c;
        // the list-reuse test leaves the same 1e-5 relative margin
        g.screen = (T)(bp.rl * bp.rl) * (T)1.00001;
    }
    if (threadIdx.x < 9) {
        g.bv[threadIdx.x] = (T)sc.bv[threadIdx.x];
        g.dh[threadIdx.x] = (T)sc.dh[threadIdx.x];
        g.D[threadIdx.x] = (T)sc.D[threadIdx.x];
    }
    if (threadIdx.x < 3) {
        g.nb[threadIdx.x] = sc.nb[threadIdx.x];
        g.m[threadIdx.x] = sc.m[threadIdx.x];
    }
}

// Writes the generalised atom force F D^T of slot t (row vector times D^T)
// and the tile's energy, virial and pair-count partials.
template <typename T>
__device__ inline void lj_finish(const LJAcc<T> &A, const LJGeom<T> &g, BandDev &b,
                                 const Tile &tl, int t, bool active) {
    if (active) {
        const T g0 = A.fx * g.D[0] + A.fy * g.D[1] + A.fz * g.D[2];
        const T g1 = A.fx * g.D[3] + A.fy * g.D[4] + A.fz * g.D[5];
        const T g2 = A.fx * g.D[6] + A.fy * g.D[7] + A.fz * g.D[8];
        const int atom = b.slot_atom[(size_t)tl.img * b.n + t];
        T *F = (T *)b.F + ((size_t)tl.img * b.rows + atom) * 3;
        F[0] = g0;
        F[1] = g1;
        F[2] = g2;
    }
    // U_i = 1/2 sum_j [4 eps (sr12 - sr6) - phi(rc)];  V = -1/2 sum r (x) f,
    // written as the symmetric virial in row-major order
    T acc[12];
    acc[0] = (T)0.5 * (g.e4 * A.e - g.ephi * (T)A.cnt);
    acc[1] = (T)(-0.5) * A.v00;
    acc[2] = acc[4] = (T)(-0.5) * A.v01;
    acc[3] = acc[7] = (T)(-0.5) * A.v02;
    acc[5] = (T)(-0.5) * A.v11;
    acc[6] = acc[8] = (T)(-0.5) * A.v12;
    acc[9] = (T)(-0.5) * A.v22;
    acc[10] = (T)A.cnt;
    acc[11] = (T)0;
    block_sum_store<12, T>(acc, b.atom_part + ((size_t)tl.img * b.atpi + tl.t) * NPART);
}

// Direct path (bands without a neighbour list: no skin, or more atoms per
// image than a list entry can index): one thread per atom in slot order
// walks the cell-list stencil and evaluates every candidate inside rc.
template <typename T>
__global__ void __launch_bounds__(TILE, sizeof(T) == 4 ? 8 : 4) k_lj(const Tile *tiles, BandDev *bands) {
    using T4 = typename Vec4<T>::type;
    Tile tl = tiles[blockIdx.x];
    BandDev &b = bands[tl.band];
    if (b.lj_cap > 0) return;  // uniform over the block: the list path runs
    const ImgScalars &sc = b.sc[tl.img];
    __shared__ LJGeom<T> g;
    lj_stage(g, sc, *b.bp);
    __syncthreads();
    const int n = b.n;
    const int t = tl.t * TILE + threadIdx.x;
    const size_t base = (size_t)tl.img * n;
    const T4 *off = (const T4 *)b.slot_off + base;
    const int *start = b.bin_start + (size_t)tl.img * (b.nbins_cap + 1);
    const T rc2 = g.rc2, sig2 = g.sig2, c24 = g.c24;
    LJAcc<T> A;
    if (t < n) {
        const T4 oi = off[t];
        lj_walk<T>(off, start, oi, b.slot_bin[base + t], g.bv, g.dh, g.nb, g.m,
                   [&](int, T ux, T uy, T uz, int, int) {
                       const T r2 = ux * ux + uy * uy + uz * uz;
                       // r2 == 0 only for the atom itself at zero shift
                       if (r2 < rc2 && r2 > (T)0) A.pair(ux, uy, uz, r2, sig2, c24);
                   });
    }
    lj_finish(A, g, b, tl, t, t < n);
}

// Neighbour list of a rebuilt image (bands with a skin): one thread per atom
// walks the cell-list stencil and keeps every candidate within rl, coalesced
// as [entry][atom].  Entries inside rc at the build come first and those of
// the skin shell after them, so that the force kernel's warps mostly agree
// on which entries have a pair term.  Images that keep their cell list keep
// their list too.
template <typename T>
__device__ inline void lj_list_atom(BandDev &b, const Tile &tl, const LJGeom<T> &g, int t) {
    using T4 = typename Vec4<T>::type;
    const int n = b.n, cap = b.lj_cap;
    const size_t base = (size_t)tl.img * n;
    const T4 *off = (const T4 *)b.slot_off + base;
    const int *start = b.bin_start + (size_t)tl.img * (b.nbins_cap + 1);
    uint32_t *L = (uint32_t *)b.nbr_slot + (size_t)tl.img * cap * n + t;
    const T rc2 = g.rc2, screen = g.screen;
    // the atom itself: slot t at zero offset and wrap
    const uint32_t self =
        lj_entry(t, 2 * g.m[0] + LJ_AXIS * 2 * g.m[1], 2 * g.m[2]);
    int nin = 0, nsh = 0;
    const T4 oi = off[t];
    lj_walk<T>(off, start, oi, b.slot_bin[base + t], g.bv, g.dh, g.nb, g.m,
               [&](int q, T ux, T uy, T uz, int i01, int i2) {
                   const T r2 = ux * ux + uy * uy + uz * uz;
                   if (!(r2 < screen)) return;
                   const uint32_t e = lj_entry(q, i01, i2);
                   if (e == self) return;
                   if (nin + nsh < cap) L[(size_t)(r2 < rc2 ? nin : cap - 1 - nsh) * n] = e;
                   if (r2 < rc2) ++nin;
                   else ++nsh;
               });
    const int total = nin + nsh;
    if (total > cap) {
        // not every slot of [0, cap) holds an entry: none is read
        atomicOr(&b.bp->status, ST_NBR_OVERFLOW);
        b.nbr_cnt[base + t] = 0;
        return;
    }
    // the shell block [cap - nsh, cap) moves down behind the inner entries,
    // and the atom itself pads the list to a whole number of LJ_UNROLL
    // entries (cap is a multiple of 8; the pair term skips r = 0)
    for (int k = 0; k < nsh; ++k) L[(size_t)(nin + k) * n] = L[(size_t)(cap - nsh + k) * n];
    const int padded = (total + LJ_UNROLL - 1) / LJ_UNROLL * LJ_UNROLL;
    for (int k = total; k < padded; ++k) L[(size_t)k * n] = self;
    b.nbr_cnt[base + t] = padded;
}

template <typename T>
__global__ void __launch_bounds__(TILE) k_lj_list(const Tile *tiles, int ntiles, BandDev *bands) {
    __shared__ LJGeom<T> g;
    for (int k = blockIdx.x; k < ntiles; k += gridDim.x) {
        const Tile tl = tiles[k];
        BandDev &b = bands[tl.band];
        const ImgScalars &sc = b.sc[tl.img];
        if (b.lj_cap == 0 || !sc.rebuild) continue;  // uniform over the block
        lj_stage(g, sc, *b.bp);
        __syncthreads();
        const int t = tl.t * TILE + threadIdx.x;
        if (t < b.n) lj_list_atom<T>(b, tl, g, t);
        __syncthreads();  // g is restaged for the next tile
    }
}

// List path: F_i, U_i and the virial from slot t's list entries.  The pair
// vector of an entry is (o_j - o_i) + c with c the displacement of the
// bin centres and wrap, c = C01[i0 + LJ_AXIS i1] + C2[i2] from per-axis
// tables of the image's current bin vectors built by each block in shared
// memory.  Entries are taken LJ_UNROLL at a time (lists are padded to a
// multiple of it): a group's offsets are gathered and the next group's
// entries loaded before the group's arithmetic, so a list load's latency
// overlaps a whole group of pair terms (7 blocks per SM leave the registers
// for it: measured faster than 8 without the overlap).
// MINB: resident blocks per SM the register allocation is held to (the
// autotuner picks it with the bin width: more blocks hide more gather
// latency, fewer leave more registers for the look-ahead)
template <typename T, int MINB>
__global__ void __launch_bounds__(TILE, MINB) k_lj_nbr(const Tile *tiles, BandDev *bands) {
    using T4 = typename Vec4<T>::type;
    Tile tl = tiles[blockIdx.x];
    BandDev &b = bands[tl.band];
    if (b.lj_cap == 0) return;  // uniform over the block: the direct path runs
    const ImgScalars &sc = b.sc[tl.img];
    __shared__ LJGeom<T> g;
    __shared__ T4 s_c01[LJ_AXIS * LJ_AXIS];
    __shared__ T4 s_c2[32];
    lj_stage(g, sc, *b.bp);
    __syncthreads();
    {
        const int L0 = 2 * (2 * g.m[0] + 1), L1 = 2 * (2 * g.m[1] + 1), L2 = 2 * (2 * g.m[2] + 1);
        for (int k = threadIdx.x; k < L0 * L1; k += TILE) {
            const int i0 = k % L0, i1 = k / L0;
            const int d0 = i0 / 2 - g.m[0], d1 = i1 / 2 - g.m[1];
            const int t0 = floor_div(d0, g.nb[0]) + (i0 & 1);
            const int t1 = floor_div(d1, g.nb[1]) + (i1 & 1);
            T4 c;
            c.x = (d0 * g.bv[0] + d1 * g.bv[3]) + (t0 * g.dh[0] + t1 * g.dh[3]);
            c.y = (d0 * g.bv[1] + d1 * g.bv[4]) + (t0 * g.dh[1] + t1 * g.dh[4]);
            c.z = (d0 * g.bv[2] + d1 * g.bv[5]) + (t0 * g.dh[2] + t1 * g.dh[5]);
            c.w = (T)0;
            s_c01[i0 + LJ_AXIS * i1] = c;
        }
        for (int k = threadIdx.x; k < L2; k += TILE) {
            const int d2 = k / 2 - g.m[2];
            const int t2 = floor_div(d2, g.nb[2]) + (k & 1);
            T4 c;
            c.x = d2 * g.bv[6] + t2 * g.dh[6];
            c.y = d2 * g.bv[7] + t2 * g.dh[7];
            c.z = d2 * g.bv[8] + t2 * g.dh[8];
            c.w = (T)0;
            s_c2[k] = c;
        }
    }
    __syncthreads();
    const int n = b.n, cap = b.lj_cap;
    const int t = tl.t * TILE + threadIdx.x;
    const size_t base = (size_t)tl.img * n;
    const T4 *off = (const T4 *)b.slot_off + base;
    const T rc2 = g.rc2, sig2 = g.sig2, c24 = g.c24;
    LJAcc<T> A;
    if (t < n) {
        const uint32_t *L = (const uint32_t *)b.nbr_slot + (size_t)tl.img * cap * n + t;
        const int cnt = b.nbr_cnt[base + t];  // a multiple of LJ_UNROLL
        const T4 oi = off[t];
        uint32_t e[LJ_UNROLL];  // the current group's entries
#pragma unroll
        for (int u = 0; u < LJ_UNROLL; ++u) e[u] = cnt > 0 ? L[(size_t)u * n] : 0u;
        for (int k = 0; k < cnt; k += LJ_UNROLL) {
            L += (size_t)LJ_UNROLL * n;
            T4 oj[LJ_UNROLL];
#pragma unroll
            for (int u = 0; u < LJ_UNROLL; ++u) oj[u] = off[e[u] & 0x1FFFFu];
            uint32_t en[LJ_UNROLL];
            const bool more = k + LJ_UNROLL < cnt;
#pragma unroll
            for (int u = 0; u < LJ_UNROLL; ++u) en[u] = more ? L[(size_t)u * n] : 0u;
#pragma unroll
            for (int u = 0; u < LJ_UNROLL; ++u) {
                const T4 a = s_c01[(e[u] >> 17) & 1023u], c = s_c2[e[u] >> 27];
                const T ux = (oj[u].x - oi.x) + (a.x + c.x);
                const T uy = (oj[u].y - oi.y) + (a.y + c.y);
                const T uz = (oj[u].z - oi.z) + (a.z + c.z);
                const T r2 = ux * ux + uy * uy + uz * uz;
                // r2 == 0: a padding entry (the atom itself)
                if (r2 < rc2 && r2 > (T)0) A.pair(ux, uy, uz, r2, sig2, c24);
            }
#pragma unroll
            for (int u = 0; u < LJ_UNROLL; ++u) e[u] = en[u];
        }
    }
    lj_finish(A, g, b, tl, t, t < n);
}

template <typename T>
void launch_lj(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s) {
    if (ntiles <= 0) return;
    k_lj<T><<<ntiles, TILE, 0, s>>>(tiles, bands);
}
template <typename T>
void launch_lj_list(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s) {
    if (ntiles <= 0) return;
    // a block per tile: a build walks ~370 candidates per atom, and in a
    // batch of many bands a large share of the images rebuilds at a time
    // (a capped grid was measured slower here)
    k_lj_list<T><<<ntiles, TILE, 0, s>>>(tiles, ntiles, bands);
}
template <typename T>
void launch_lj_nbr(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s, int minb) {
    if (ntiles <= 0) return;
    if (sizeof(T) == 8) {
        k_lj_nbr<T, 4><<<ntiles, TILE, 0, s>>>(tiles, bands);
        return;
    }
    switch (minb) {
        case 5: k_lj_nbr<T, 5><<<ntiles, TILE, 0, s>>>(tiles, bands); break;
        case 6: k_lj_nbr<T, 6><<<ntiles, TILE, 0, s>>>(tiles, bands); break;
        case 8: k_lj_nbr<T, 8><<<ntiles, TILE, 0, s>>>(tiles, bands); break;
        default: k_lj_nbr<T, 7><<<ntiles, TILE, 0, s>>>(tiles, bands); break;
    }
}
template void launch_lj<float>(const Tile *, int, BandDev *, cudaStream_t);
template void launch_lj<double>(const Tile *, int, BandDev *, cudaStream_t);
template void launch_lj_list<float>(const Tile *, int, BandDev *, cudaStream_t);
template void launch_lj_list<double>(const Tile *, int, BandDev *, cudaStream_t);
template void launch_lj_nbr<float>(const Tile *, int, BandDev *, cudaStream_t, int);
template void launch_lj_nbr<double>(const Tile *, int, BandDev *, cudaStream_t, int);

}  // namespace cfneb
