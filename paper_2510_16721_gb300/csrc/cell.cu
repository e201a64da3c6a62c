// Cell filter inverse map and cell-list build.
//
// Map-back (Sec. II.C): the lattice rows of X hold c B; B = X_lat / c is
// symmetrised and D = B^(1/2) taken with a cyclic Jacobi eigen-solve in FP64
// (rotation-free variant), or D = X_lat / c (deformation-gradient variant).
// Then h = h0 D, and the bin geometry of the image is derived from the
// perpendicular widths of h.
//
// Cell list: atoms are binned in fractional space (s = R~ h0^-1, which is
// also R h^-1 since R = R~ D and h = h0 D), wrapped into [0, 1).  The bin
// edge vectors bv_a = h_a / nb_a are rounded to T, and each atom stores its
// Cartesian offset from the centre of its bin, sum_a (b_a + 1/2) bv_a, in T.
// A pair vector is then (off_j - off_i) + sum_a (delta_a bv_a + t_a dh_a),
// where delta is the unwrapped bin offset of the neighbour bin, t its
// periodic shift and dh_a = h_a - nb_a bv_a the (tiny) difference between a
// lattice vector and nb_a rounded bin vectors.  For |delta| <= 1 in an
// orthorhombic cell every term is exact in FP32, so the only roundings are
// those of the two small offsets and of the final sums: pair vectors keep
// ~6e-8 A absolute accuracy whatever the cell size.  Enumerating delta over
// [-m_a, m_a] with m_a = ceil(rc / bin width) visits every periodic image
// of every atom within rc exactly once, also when rc exceeds half the cell
// width (no minimum-image assumption; the neighbourhoods of Sec. II.B are
// periodic).
//
// Determinism: atoms are counted into bins with integer atomics, then each
// bin's atoms are ordered by atom index, so the slot order (and every
// summation order downstream) is the same on every run.
//
// Reuse with a skin: with skin > 0 the stencil and any neighbour list cover
// rl = rc + skin, and an image keeps its bins (and lists) while they still
// hold every pair inside rc.  With R = R~ D, a pair vector is rho D where
// rho is its R~-frame vector; from the build (D_b) to now (D), a pair that
// was at |r_b| >= rl is now at least rl (1 - |D_b^-1 D - I|) - 2 d |D| away,
// d being the largest displacement |R~ - R~_b| of any atom.  While that
// bound stays above rc the bins of the build are kept: each atom's offset is
// recomputed from its current position against the centre of its old bin
// (the pair-vector identity above holds for any position, inside the bin or
// not), which costs one pass over the atoms instead of a rebuild.
#include <algorithm>

#include "common.cuh"

namespace cfneb {

// ---- 3x3 symmetric square root -----------------------------------------
//
// On this GPU a dependent FP64 operation costs ~64 cycles and an FP64
// divide or square root several hundred, and the map-back of every image is
// on the critical path of each step.  The symmetric root is therefore taken
// with the coupled Newton-Schulz iteration (Higham, Functions of Matrices,
// 2008, Sec. 6.7), which needs matrix products only: with Y0 = B/mu, Z0 = I
// and T = (3I - Z Y)/2, Y <- Y T and Z <- T Z converge quadratically to
// (B/mu)^(1/2) and (B/mu)^(-1/2) when the eigenvalues of B/mu lie in (0, 2).
// Every iterate is a polynomial in B, so Y and Z stay symmetric and commute
// with B.  mu is the midpoint of a bracket of the spectrum: g, the largest
// Gershgorin row bound (>= lambda_max), and det B / g^2 (<= lambda_min).
// The products run lane-parallel (k_mapback).

// Bin grid of an image with cell h (one thread): the bin counts nb and
// stencil half widths m from the perpendicular widths and the list cutoff.
// Between rebuilds the grid stays as built and only the bin vectors follow
// the cell (bin_vectors_warp).
__device__ void bin_grid(const BandParams *bp, int nbins_cap, const double *h, double omega,
                         ImgScalars &sc) {
    const double rl = bp->rl > 0.0 ? bp->rl : bp->rc;
    int nb[3];
    float w[3];
    // perpendicular widths w_a = Omega / |h_b x h_c| (only choose the bin
    // grid: FP32, shaded down by 1e-4 so the stencil is never too narrow,
    // also for atoms binned in FP32)
    for (int a = 0; a < 3; ++a) {
        const double *u = h + 3 * ((a + 1) % 3), *v = h + 3 * ((a + 2) % 3);
        const double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2],
                     cz = u[0] * v[1] - u[1] * v[0];
        w[a] = (float)omega / sqrtf((float)(cx * cx + cy * cy + cz * cz)) * 0.9999f;
    }
    for (int a = 0; a < 3; ++a) {
        // the innermost axis may be binned finer: the LJ kernel walks it
        // as contiguous rows, so finer bins there trim the candidate
        // range without adding rows
        const float bw = (float)bp->bin_w / (a == 2 ? (float)bp->row_refine : 1.0f);
        // never so fine that the stencil would need more than
        // MAX_STENCIL bins per side (coarser bins are always correct)
        const float q = fminf(floorf(w[a] / bw),
                              floorf(w[a] * (float)MAX_STENCIL / (float)rl * 0.9999f));
        nb[a] = q < 1.0f ? 1 : (q > 1024.0f ? 1024 : (int)q);
    }
    // keep within the bin capacity: coarser bins are always correct
    while ((long long)nb[0] * nb[1] * nb[2] > nbins_cap) {
        int a = (nb[0] >= nb[1] && nb[0] >= nb[2]) ? 0 : (nb[1] >= nb[2] ? 1 : 2);
        nb[a] -= 1;
    }
    for (int a = 0; a < 3; ++a) {
        const float bw = w[a] / nb[a];
        const int m = (int)ceilf((float)rl / bw);
        // a cell narrower than rl / MAX_STENCIL: periodic images beyond the
        // stencil would be missed
        if (m > MAX_STENCIL) atomicOr(const_cast<int *>(&bp->status), ST_NBR_OVERFLOW);
        sc.m[a] = m < 1 ? 1 : (m > MAX_STENCIL ? MAX_STENCIL : m);
        sc.nb[a] = nb[a];
    }
    sc.nbins = nb[0] * nb[1] * nb[2];
}

// The rebuild decision of one image on its staged record sc (one thread):
// keep the bins of the build while the bound in the header comment holds,
// else rebuild (always when forced, when the band's images were rearranged,
// or while autotuning).  d = the largest displacement since the build; the
// cell's part of the bound (skin_terms) is current in sc.
__device__ void skin_decide_one(const BandParams *bp, int nbins_cap, ImgScalars &sc, double d,
                                int force) {
    bool rebuild = force || bp->stale || bp->tune_rebuild || sc.builds == 0;
    if (!rebuild) {
        const double bound = bp->rl * (1.0 - 1e-5) * (1.0 - (double)sc.skin_e) -
                             2.0 * d * (double)sc.skin_nD * (1.0 + 1e-5);
        rebuild = !(bound > bp->rc);
    }
    if (rebuild) {
        bin_grid(bp, nbins_cap, sc.h, sc.omega, sc);
        float Db[9];
        for (int k = 0; k < 9; ++k) {
            sc.Db[k] = sc.D[k];
            Db[k] = (float)sc.D[k];
        }
        inv3f(Db, sc.Dbif);
        skin_terms(sc, sc.Dbif);
        sc.builds += 1;
    }
    sc.rebuild = rebuild ? 1 : 0;
    sc.dmax = d;
    sc.evals += 1;
}

// Map-back of one image per warp and its cell-list decision.  The cell
// (image_cell_warp: D, h, Omega and the bin vectors) is taken over from the
// last move when k_fire_update already computed it for the current lattice
// rows; it is computed here for forced evaluations, after the band's images
// were rearranged or reloaded (stale) and whenever the move did not leave
// it.  Then with no skin a rebuild on the new cell, with a skin the reuse
// test on the displacements the last move left per row tile.  The image
// record is staged in shared memory, updated and written back whole.
template <typename T>
__global__ void __launch_bounds__(32) k_mapback(const ImgRef *imgs, int count, BandDev *bands,
                                                int force) {
    const ImgRef r = imgs[blockIdx.x];
    BandDev &b = bands[r.band];
    __shared__ BandParams s_bp;
    __shared__ ImgScalars s_sc;
    stage_copy(&s_bp, b.bp);
    stage_copy(&s_sc, &b.sc[r.img]);
    __syncwarp();
    const BandParams *bp = &s_bp;
    ImgScalars &sc = s_sc;
    const int lane = threadIdx.x & 31;
    const bool fresh = !force && !bp->stale && sc.cell_fresh;
    double h = 0.0;
    if (!fresh) {
        const T *Xl = (const T *)b.X + ((size_t)r.img * b.rows + b.n) * 3;
        const bool ok = image_cell_warp(cell_in(bp), (double)Xl[lane % 9], sc, h);
        if (!ok && lane == 0) atomicOr(&b.bp->status, ST_NOT_SPD);
    }
    // largest displacement since the last build (skin > 0), in FP32 (a max
    // is exact in any precision)
    double dmax = 0.0;
    if (b.skin_part) {
        // per row tile, left by the last move (k_fire_update)
        const float *part = b.skin_part + (size_t)r.img * b.atpi;
        float m = 0.0f;
#pragma unroll 8
        for (int t = lane; t < b.rtpi; t += 32) m = fmaxf(m, part[t]);
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        dmax = (double)m;
    }
    __syncwarp();
    if (lane == 0) {
        sc.cell_fresh = 1;
        if (!fresh && bp->skin > 0.0) skin_terms(sc, sc.Dbif);
        if (bp->skin <= 0.0) {
            // no skin: the cell list is rebuilt at every evaluation
            bin_grid(bp, b.nbins_cap, sc.h, sc.omega, sc);
            sc.rebuild = 1;
            sc.builds += 1;
            sc.evals += 1;
        } else {
            skin_decide_one(bp, b.nbins_cap, sc, dmax, force);
        }
    }
    __syncwarp();
    // the grid (new or kept) follows the cell; a move that left the cell
    // also left the bin vectors of the kept grid
    if (!fresh || sc.rebuild) bin_vectors_warp(sc, sc.nb[(lane % 9) / 3], sc.h[lane % 9]);
    __syncwarp();
    stage_copy(&b.sc[r.img], &s_sc);
}

// Offset of an atom from the centre of its (kept) bin, R - K with R = R~ D
// and K = sum_a (wrap_a h_a + (b_a + 1/2) bv_a), as a leading part and a
// remainder.  FP64 path: in FP64.  FP32 path: in pairs of FP32 (products
// split exactly with FMA, sums with Knuth's two-sum), from the FP32 pairs
// of D and h that k_mapback stores; bv is exact in FP32 by construction.
// Both keep the offset to ~1e-14 relative of the cell size, far below the
// FP32 leading part's rounding.
__device__ inline void refresh_offset(const ImgScalars &sc, const BandParams *bp, const double *X,
                                      const int *wr, const int *bi, double4_32a &o,
                                      double4_32a &lo) {
    double off[3];
    double s[3];
    for (int a = 0; a < 3; ++a)
        s[a] = (X[0] * bp->h0inv[a] + X[1] * bp->h0inv[3 + a] + X[2] * bp->h0inv[6 + a]) -
               (double)wr[a];
    for (int c = 0; c < 3; ++c) {
        const double R = s[0] * sc.h[c] + s[1] * sc.h[3 + c] + s[2] * sc.h[6 + c];
        const double ctr = (bi[0] + 0.5) * sc.bv[c] + (bi[1] + 0.5) * sc.bv[3 + c] +
                           (bi[2] + 0.5) * sc.bv[6 + c];
        off[c] = R - ctr;
    }
    o.x = off[0];
    o.y = off[1];
    o.z = off[2];
    o.w = (double)bi[2];
    lo.x = lo.y = lo.z = lo.w = 0.0;
}

struct F2 {  // unevaluated sum hi + lo of two floats
    float hi, lo;
};
// a (hi + lo) exactly up to the rounding of the low product
__device__ inline F2 f2_mul(float a, float bh, float bl) {
    const float p = __fmul_rn(a, bh);
    float e = fmaf(a, bh, -p);
    e = fmaf(a, bl, e);
    return {p, e};
}
__device__ inline F2 f2_add(F2 a, F2 b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float hi = __fadd_rn(s, e);
    return {hi, __fsub_rn(e, __fsub_rn(hi, s))};
}

// Many-body (Tersoff, NEP-style) bands: the leading part is rounded to a
// multiple of 2^-20 A (the remainder goes to the low part, exactly), so that
// the force kernel forms (o_j - o_i) + (bin displacement) exactly with plain
// FP32 operations: every term sits on the 2^-20 grid (bin vectors on a
// coarser power-of-two grid) and the sums stay below 2^3 A.
constexpr float OFF_GRID = 1048576.0f;  // 2^20

__device__ inline F2 f2_prod(float a, float b) {  // a b exactly
    const float p = __fmul_rn(a, b);
    return {p, fmaf(a, b, -p)};
}

// K = sum_a (wrap_a h_a + (b_a + 1/2) bv_a) is formed as
// sum_a m_a bv_a + sum_a wrap_a dh_a with m_a = wrap_a nb_a + b_a + 1/2
// (h_a = nb_a bv_a + dh_a): each m_a bv_a is exact as a pair (bv exact in
// FP32, m_a a half-integer far below 2^23), the dh terms are tiny and join
// the low part.
__device__ inline void refresh_offset(const ImgScalars &sc, const BandParams *bp, const float *X,
                                      const int *wr, const int *bi, float4 &o, float4 &lo) {
    const float *Dh = sc.dfl, *Dl = sc.dfl + 9;
    float m[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) m[a] = (float)(wr[a] * sc.nb[a] + bi[a]) + 0.5f;
    float off[2][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        // R_c = sum_k X_k D_kc (X exact in FP32)
        F2 R = f2_mul(X[0], Dh[c], Dl[c]);
        R = f2_add(R, f2_mul(X[1], Dh[3 + c], Dl[3 + c]));
        R = f2_add(R, f2_mul(X[2], Dh[6 + c], Dl[6 + c]));
        F2 K = f2_prod(m[0], sc.bvf[c]);
        K = f2_add(K, f2_prod(m[1], sc.bvf[3 + c]));
        K = f2_add(K, f2_prod(m[2], sc.bvf[6 + c]));
        K.lo = fmaf((float)wr[0], sc.dhf[c],
                    fmaf((float)wr[1], sc.dhf[3 + c], fmaf((float)wr[2], sc.dhf[6 + c], K.lo)));
        const F2 d = f2_add(R, {-K.hi, -K.lo});
        if (bp->kind != KIND_LJ) {
            const float q = rintf(d.hi * OFF_GRID) * (1.0f / OFF_GRID);
            off[0][c] = q;
            off[1][c] = __fadd_rn(__fsub_rn(d.hi, q), d.lo);  // d.hi - q is exact
        } else {
            off[0][c] = d.hi;
            off[1][c] = d.lo;
        }
    }
    o = make_float4(off[0][0], off[0][1], off[0][2], (float)bi[2]);
    lo = make_float4(off[1][0], off[1][1], off[1][2], 0.0f);
}

// Bin and periodic wrap of an atom: s = R~ h0^-1 wrapped into [0, 1).  FP64
// path in FP64; FP32 path in FP32 (a bin choice off by FP32 rounding near a
// bin face puts the atom ~1e-7 of the cell outside its bin, inside the
// 1e-4 margin the stencil widths are shaded by; the offset itself is exact).
__device__ inline void bin_of(const ImgScalars &sc, const BandParams *bp, const double *X, int *bi,
                              int *wrap) {
    for (int a = 0; a < 3; ++a) {
        double s = X[0] * bp->h0inv[a] + X[1] * bp->h0inv[3 + a] + X[2] * bp->h0inv[6 + a];
        const double fl = floor(s);
        s -= fl;
        wrap[a] = (int)fl;
        if (s >= 1.0) {
            s = 0.0;
            wrap[a] += 1;
        }
        // any bin index outside [0, nb) (a non-finite coordinate) goes to an
        // edge bin: the index stays in range whatever the input
        const int q = (int)(s * sc.nb[a]);
        bi[a] = q >= sc.nb[a] ? sc.nb[a] - 1 : (q < 0 ? 0 : q);
    }
}
__device__ inline void bin_of(const ImgScalars &sc, const BandParams *, const float *X, int *bi,
                              int *wrap) {
    const float *hi = sc.dfl + 36;  // h0^-1 in FP32
    for (int a = 0; a < 3; ++a) {
        float s = X[0] * hi[a] + X[1] * hi[3 + a] + X[2] * hi[6 + a];
        const float fl = floorf(s);
        s -= fl;
        wrap[a] = (int)fl;
        if (s >= 1.0f) {
            s = 0.0f;
            wrap[a] += 1;
        }
        const int q = (int)(s * (float)sc.nb[a]);
        bi[a] = q >= sc.nb[a] ? sc.nb[a] - 1 : (q < 0 ? 0 : q);
    }
}

// In a graph (has_cond), the first tile of every image that rebuilds also
// switches on the conditional node that holds the rebuild kernels (its
// value is reset to 0 at every launch of the graph).
template <typename T>
__global__ void __launch_bounds__(TILE) k_bin_assign(const Tile *tiles, BandDev *bands,
                                                     cudaGraphConditionalHandle cond,
                                                     int has_cond) {
    using T4 = typename Vec4<T>::type;
    Tile tl = tiles[blockIdx.x];
    BandDev &b = bands[tl.band];
    const ImgScalars &sc = b.sc[tl.img];
    const BandParams *bp = b.bp;
    if (has_cond && sc.rebuild && tl.t == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 1u);
    if (!sc.rebuild) {
        // keep the bins of the build: thread = slot, offset from the centre
        // of the slot's bin at the current position (unwrapped as at the build)
        const int t = tl.t * TILE + threadIdx.x;
        if (t >= b.n) return;
        const size_t st = (size_t)tl.img * b.n + t;
        const int i = b.slot_atom[st];
        int bi[3];
        unpack_bin(b.slot_bin[st], bi[0], bi[1], bi[2]);
        const int *wr = b.atom_wrap + ((size_t)tl.img * b.n + i) * 3;
        const T *Xi = (const T *)b.X + ((size_t)tl.img * b.rows + i) * 3;
        T4 o, lo;
        refresh_offset(sc, bp, Xi, wr, bi, o, lo);
        ((T4 *)b.slot_off)[st] = o;
        ((T4 *)b.slot_off_lo)[st] = lo;
        return;
    }
    int i = tl.t * TILE + threadIdx.x;
    if (i >= b.n) return;
    const T *Xi = (const T *)b.X + ((size_t)tl.img * b.rows + i) * 3;
    int bi[3], wrap[3];
    bin_of(sc, bp, Xi, bi, wrap);
    int lin = (bi[0] * sc.nb[1] + bi[1]) * sc.nb[2] + bi[2];
    size_t ai = (size_t)tl.img * b.n + i;
    int rank = atomicAdd(&b.bin_count[(size_t)tl.img * b.nbins_cap + lin], 1);
    b.atom_bin[ai] = lin;
    b.atom_rank[ai] = rank;
    // offset from the bin centre (the w lane holds the innermost bin index,
    // for the row traversal of the LJ kernel)
    T4 o, lo;
    refresh_offset(sc, bp, Xi, wrap, bi, o, lo);
    ((T4 *)b.atom_off)[ai] = o;
    ((T4 *)b.atom_off_lo)[ai] = lo;
    if (b.ref_X) {  // a skin: reference state of the build (row layout of X)
        T *ref = (T *)b.ref_X + ((size_t)tl.img * b.rows + i) * 3;
        ref[0] = Xi[0];
        ref[1] = Xi[1];
        ref[2] = Xi[2];
        for (int a = 0; a < 3; ++a) b.atom_wrap[ai * 3 + a] = wrap[a];
    }
}

// Exclusive scan of the bin counts, in three passes over SCAN_TILE-bin
// tiles: tile sums, a scan of the tile sums per image, and a block-wide scan
// of each tile offset by its tile prefix.  Integer arithmetic: exact and
// deterministic.  Counts are reset to zero for the next build.
constexpr int SCAN_TILE = 1024;

__device__ inline int block_excl_scan_1024(int v, int *total) {
    __shared__ int wsum[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        wsum[lane] = s;  // inclusive scan of the warp sums
    }
    __syncthreads();
    const int before = (w > 0) ? wsum[w - 1] : 0;
    *total = wsum[31];
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(256) k_bin_tilesum(const ImgRef *imgs, BandDev *bands) {
    ImgRef r = imgs[blockIdx.y];
    BandDev &b = bands[r.band];
    if (!b.sc[r.img].rebuild) return;
    const int nb = b.sc[r.img].nbins;
    const int *cnt = b.bin_count + (size_t)r.img * b.nbins_cap;
    __shared__ int ws[8];
    // a fixed grid strides over the tiles: images that keep their cell list
    // cost one read per block
    for (int c = blockIdx.x; c * SCAN_TILE < nb; c += gridDim.x) {
        const int t0 = c * SCAN_TILE;
        int s = 0;
        for (int k = threadIdx.x; k < SCAN_TILE && t0 + k < nb; k += blockDim.x) s += cnt[t0 + k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot += ws[q];
            b.bin_tsum[(size_t)r.img * b.tsum_cap + c] = tot;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) k_bin_tilescan(const ImgRef *imgs, BandDev *bands) {
    ImgRef r = imgs[blockIdx.x];
    BandDev &b = bands[r.band];
    if (!b.sc[r.img].rebuild) return;
    const int nt = (b.sc[r.img].nbins + SCAN_TILE - 1) / SCAN_TILE;
    int *ts = b.bin_tsum + (size_t)r.img * b.tsum_cap;
    int carry = 0;
    for (int base = 0; base < nt; base += 1024) {
        const int k = base + threadIdx.x;
        const int v = k < nt ? ts[k] : 0;
        int tot;
        const int ex = block_excl_scan_1024(v, &tot);
        if (k < nt) ts[k] = carry + ex;
        carry += tot;
    }
}

__global__ void __launch_bounds__(1024) k_bin_scanfill(const ImgRef *imgs, BandDev *bands) {
    ImgRef r = imgs[blockIdx.y];
    BandDev &b = bands[r.band];
    if (!b.sc[r.img].rebuild) return;
    const int nb = b.sc[r.img].nbins;
    int *cnt = b.bin_count + (size_t)r.img * b.nbins_cap;
    int *start = b.bin_start + (size_t)r.img * (b.nbins_cap + 1);
    for (int c = blockIdx.x; c * SCAN_TILE < nb; c += gridDim.x) {
        const int bin = c * SCAN_TILE + threadIdx.x;
        const int v = bin < nb ? cnt[bin] : 0;
        int tot;
        const int ex = block_excl_scan_1024(v, &tot);
        const int off = b.bin_tsum[(size_t)r.img * b.tsum_cap + c];
        if (bin < nb) {
            start[bin] = off + ex;
            cnt[bin] = 0;
            if (bin == nb - 1) start[nb] = off + ex + v;
        }
    }
}

__global__ void __launch_bounds__(TILE) k_bin_scatter(const Tile *tiles, int ntiles, BandDev *bands) {
    for (int k = blockIdx.x; k < ntiles; k += gridDim.x) {
        const Tile tl = tiles[k];
        BandDev &b = bands[tl.band];
        if (!b.sc[tl.img].rebuild) continue;
        const int i = tl.t * TILE + threadIdx.x;
        if (i >= b.n) continue;
        const size_t ai = (size_t)tl.img * b.n + i;
        const int *start = b.bin_start + (size_t)tl.img * (b.nbins_cap + 1);
        b.slot_unsorted[(size_t)tl.img * b.n + start[b.atom_bin[ai]] + b.atom_rank[ai]] = i;
    }
}

// Threads stride over the bins: order each bin's atoms by atom index and
// write the sorted slot arrays.
template <typename T>
__global__ void k_bin_order(const ImgRef *imgs, BandDev *bands) {
    using T4 = typename Vec4<T>::type;
    ImgRef r = imgs[blockIdx.y];
    BandDev &b = bands[r.band];
    if (!b.sc[r.img].rebuild) return;
    const int nbins = b.sc[r.img].nbins;
    const int *start = b.bin_start + (size_t)r.img * (b.nbins_cap + 1);
    const size_t base = (size_t)r.img * b.n;
    const int *un = b.slot_unsorted + base;
    const int nb1 = b.sc[r.img].nb[1], nb2 = b.sc[r.img].nb[2];
    for (int bin = blockIdx.x * blockDim.x + threadIdx.x; bin < nbins;
         bin += gridDim.x * blockDim.x) {
        const int s0 = start[bin], s1 = start[bin + 1];
        const int b0 = bin / (nb1 * nb2), b1 = (bin / nb2) % nb1;
        const int pb = pack_bin(b0, b1, bin % nb2);
        for (int p = s0; p < s1; ++p) {
            const int idx = un[p];
            int rk = 0;
            for (int q = s0; q < s1; ++q) rk += (un[q] < idx);
            const int dst = s0 + rk;
            b.slot_atom[base + dst] = idx;
            b.slot_bin[base + dst] = pb;
            b.atom_slot[base + idx] = dst;
            ((T4 *)b.slot_off)[base + dst] = ((const T4 *)b.atom_off)[base + idx];
            ((T4 *)b.slot_off_lo)[base + dst] = ((const T4 *)b.atom_off_lo)[base + idx];
        }
    }
}

// Cartesian positions R = R~ D (FP64) of the listed images, for output.
template <typename T>
__global__ void k_cartesian(const ImgRef *imgs, BandDev *bands) {
    ImgRef r = imgs[blockIdx.y];
    BandDev &b = bands[r.band];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.n) return;
    const ImgScalars &sc = b.sc[r.img];
    const T *Xi = (const T *)b.X + ((size_t)r.img * b.rows + i) * 3;
    double x[3] = {(double)Xi[0], (double)Xi[1], (double)Xi[2]};
    double *o = b.cart + ((size_t)r.img * b.n + i) * 3;
    for (int c = 0; c < 3; ++c) o[c] = x[0] * sc.D[c] + x[1] * sc.D[3 + c] + x[2] * sc.D[6 + c];
}

// ---- launchers -------------------------------------------------------------

template <typename T>
void launch_mapback(const ImgRef *imgs, int count, BandDev *bands, int force, cudaStream_t s) {
    if (count <= 0) return;
    k_mapback<T><<<count, 32, 0, s>>>(imgs, count, bands, force);
}
template <typename T>
void launch_bin_assign(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s,
                       cudaGraphConditionalHandle cond, int has_cond) {
    if (ntiles <= 0) return;
    k_bin_assign<T><<<ntiles, TILE, 0, s>>>(tiles, bands, cond, has_cond);
}
void launch_bin_scan(const ImgRef *imgs, int count, int max_bins, BandDev *bands,
                     cudaStream_t s, int part) {
    if (count <= 0 || max_bins <= 0) return;
    dim3 grid(std::min((max_bins + SCAN_TILE - 1) / SCAN_TILE, 32), count);
    if (part == 0) k_bin_tilesum<<<grid, 256, 0, s>>>(imgs, bands);
    else if (part == 1) k_bin_tilescan<<<count, 1024, 0, s>>>(imgs, bands);
    else k_bin_scanfill<<<grid, 1024, 0, s>>>(imgs, bands);
}
void launch_bin_scatter(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s) {
    if (ntiles <= 0) return;
    k_bin_scatter<<<ntiles < gated_grid() ? ntiles : gated_grid(), TILE, 0, s>>>(tiles, ntiles, bands);
}
template <typename T>
void launch_bin_order(const ImgRef *imgs, int count, int max_bins, BandDev *bands,
                      cudaStream_t s) {
    if (count <= 0 || max_bins <= 0) return;
    dim3 grid(std::min((max_bins + 127) / 128, 128), count);
    k_bin_order<T><<<grid, 128, 0, s>>>(imgs, bands);
}
template <typename T>
void launch_cartesian(const ImgRef *imgs, int count, int max_n, BandDev *bands, cudaStream_t s) {
    if (count <= 0 || max_n <= 0) return;
    dim3 grid((max_n + 127) / 128, count);
    k_cartesian<T><<<grid, 128, 0, s>>>(imgs, bands);
}

#define CFNEB_INST(T)                                                                     \
    template void launch_mapback<T>(const ImgRef *, int, BandDev *, int, cudaStream_t);  \
    template void launch_bin_assign<T>(const Tile *, int, BandDev *, cudaStream_t,       \
                                       cudaGraphConditionalHandle, int);                 \
    template void launch_bin_order<T>(const ImgRef *, int, int, BandDev *, cudaStream_t); \
    template void launch_cartesian<T>(const ImgRef *, int, int, BandDev *, cudaStream_t);
CFNEB_INST(float)
CFNEB_INST(double)
#undef CFNEB_INST

}  // namespace cfneb
