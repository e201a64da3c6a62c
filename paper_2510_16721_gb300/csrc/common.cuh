// Shared device-side data layout of the CFNEB library.
//
// A band of N images of n atoms lives in HBM as image-major arrays:
//   X, F, Fneb, v : [ncap][n+3][3] of T   (T = double for CFNEB_FP64,
//                                           float for CFNEB_MIXED)
// rows 0..n-1 are atoms (R~ and the forces conjugate to it), rows n..n+2 the
// lattice coordinate c B (Sec. II.C: the (n+3) "atoms" of the cell filter).
// Per-image FP64 scalars (energy, virial, D, h, bin geometry) sit in
// ImgScalars[ncap]; per-band constants and FIRE state in BandParams.
//
// Kernels are launched over tile tables: each tile is (band, image, t) and
// covers atoms [t*TILE, (t+1)*TILE) (atom tiles, one thread per atom) or
// rows [t*RTILE, (t+1)*RTILE) (row tiles of the band-vector kernels, RPT
// rows per thread) of that image, so any mix of bands of different sizes
// runs in one launch.  Partial sums of a tile land in a
// fixed slot (image, t) of its band, and every reduction sums the slots of a
// band in slot order: results do not depend on which other bands share the
// launch.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <stdint.h>

namespace cfneb {

constexpr int TILE = 128;           // atoms per atom tile = threads per block
constexpr int RTHREADS = 256;       // threads per block of the row-tile kernels
constexpr int RPT = 4;              // consecutive rows per thread of the row-tile kernels
constexpr int RTILE = RTHREADS * RPT;  // rows per row tile (band vector kernels)
constexpr int MAXN_TERSOFF = 16;    // Tersoff list capacity per atom (entries within rl)
constexpr int NPART = 12;           // doubles per tile partial record
constexpr int MAX_STENCIL = 7;      // |delta| <= 7 bins per axis
// NEP-style potential: Chebyshev basis size, radial and angular functions,
// largest Legendre order, hidden units; descriptor and weight counts
constexpr int NEP_K = 6, NEP_NR = 4, NEP_NA = 2, NEP_L = 4, NEP_H = 16;
constexpr int NEP_ND = NEP_NR + NEP_NA * NEP_L;
constexpr int NEP_NW = NEP_NR * NEP_K + NEP_NA * NEP_K + NEP_H * NEP_ND + 2 * NEP_H + 1;
// offsets of cR, cA, W0, b0, w1, b1 in the flat weight array
constexpr int NEP_OCR = 0, NEP_OCA = NEP_NR * NEP_K, NEP_OW0 = NEP_OCA + NEP_NA * NEP_K,
              NEP_OB0 = NEP_OW0 + NEP_H * NEP_ND, NEP_OW1 = NEP_OB0 + NEP_H,
              NEP_OB1 = NEP_OW1 + NEP_H;
constexpr int LJ_LIST_MAX_ATOMS = 1 << 17;  // LJ list entries index 17-bit slots
// SMs of the current device (cached per device)
inline int sm_count() {
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (!cached[dev]) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            sms <= 0)
            sms = 152;
        cached[dev] = sms;
    }
    return cached[dev];
}
// Grid of the kernels that only do work for images rebuilding their lists:
// a fixed grid (8 blocks per SM of the current device) strides over the
// tiles, so a step in which most images keep their lists costs a few reads
// per block instead of a block per tile.
inline int gated_grid() { return sm_count() * 8; }

// potential kinds of BandParams::kind (the values of include/cfneb.h)
constexpr int KIND_LJ = 0, KIND_TERSOFF = 1, KIND_NEP = 2;

// device status bits (BandParams::status)
enum : int {
    ST_NOT_SPD = 1,
    ST_NBR_OVERFLOW = 2,
    ST_NONFINITE = 4,
};

struct ImgScalars {
    double E;            // energy (U + P Omega) of the last step's evaluation
    double U;            // potential energy
    double E64;          // FP64 energy (U + P Omega) for reporting
    double V[9];         // virial, V_eff = V - P Omega I
    double D[9];         // deformation gradient (symmetric root of B)
    double Dinv[9];
    double h[9];         // current cell h = h0 D (rows = lattice vectors)
    double hinv[9];
    double bv[9];        // bin edge vectors, row a = h_a / nb_a rounded to T
    double dh[9];        // wrap correction, row a = h_a - nb_a bv_a
    double omega;        // |det h|
    double dots[10];     // |dX+|^2, |dX-|^2, dX+.dX-, F.dX+, F.dX-, F.F, F.v,
                         // v.v, dX+.v, dX-.v (band pass 1)
    double coef[2];      // f_NEB = F + coef[0] dX+ + coef[1] dX-
    double fire[3];      // this image's F_NEB.v, |F_NEB|^2, |v|^2
    double pairs;        // neighbour entries inside the cutoff (last evaluation)
    double triples;      // ordered neighbour pairs (j, k != j) of the atoms (Tersoff)
    double Db[9];        // D when the cell list was last built (skin test)
    double dmax;         // largest |R~ - R~ at the build| of this evaluation
    long long builds;    // cell-list builds of this image slot
    long long evals;     // evaluations of this image slot
    float dfl[45];       // FP32: D hi, D lo, h hi, h lo (pairs), h0^-1 (cell list)
    float bvf[9];        // bv in FP32 (exact: bv has at most 20 significant bits)
    float dhf[9];        // dh in FP32 (the offset refresh's wrap term)
    float Dbif[9];       // FP32 inverse of Db (list reuse)
    float skin_e, skin_nD;  // the cell's part of the reuse bound (skin_terms)
    int nb[3];           // bins per axis
    int m[3];            // stencil half width per axis
    int nbins;
    int rebuild;         // this evaluation rebuilds the cell list
    unsigned int done;   // row tiles of this image finished in band pass 1
    int cell_fresh;      // D, h, Omega and the bin vectors follow the current
                         // lattice rows (set by the map-back and by the move)
};

struct TersoffParams {
    double A, B, lambda1, lambda2, beta, n, c, d, h, R, D;
};

template <typename T>
struct __align__(8) TP {  // Tersoff constants in T (derived once per band, on the host)
    T A, B, l1, l2, beta, n, c2, d2, h, R, D, Rhi, pi_2D, pi_4D, inv2n, c2d2;
    T AeR, BeR;        // A exp(-l1 R), B exp(-l2 R)
    T R2hi, R2lo;      // R^2 as a two-term sum
    T Dlo;             // D - (T)D
    T pad_;            // (a whole number of 8-byte words: staged by word copies)
    // host only (std::exp of the host library): the device reads the result
    __host__ void load(const TersoffParams &p) {
        A = (T)p.A; B = (T)p.B; l1 = (T)p.lambda1; l2 = (T)p.lambda2; beta = (T)p.beta;
        n = (T)p.n; c2 = (T)(p.c * p.c); d2 = (T)(p.d * p.d); h = (T)p.h; R = (T)p.R;
        D = (T)p.D; Rhi = (T)(p.R + p.D);
        pi_2D = (T)(0.5 * 3.14159265358979323846 / p.D);
        pi_4D = (T)(0.25 * 3.14159265358979323846 / p.D);
        inv2n = (T)(0.5 / p.n);
        c2d2 = (T)(p.c * p.c / (p.d * p.d));
        AeR = (T)(p.A * std::exp(-p.lambda1 * p.R));
        BeR = (T)(p.B * std::exp(-p.lambda2 * p.R));
        R2hi = (T)(p.R * p.R);
        R2lo = (T)(p.R * p.R - (double)R2hi);
        Dlo = (T)(p.D - (double)D);
    }
};


struct BandParams {
    // constants of the band
    double h0[9], h0inv[9];
    double c;            // cell factor: X_lat = c B
    double pressure;
    double k;            // spring constant
    double dt0, dt_max, maxstep;
    double rc;           // potential cutoff
    double skin;         // neighbour-list skin (0: rebuild every evaluation)
    double rl;           // list cutoff rc + skin (0 in records made before skins: rc)
    double bin_w;        // target bin width
    double ftol;         // convergence tolerance (< 0: never converged)
    double pot[12];      // LJ: eps, sigma, rc, phi(rc) or 0; Tersoff: A, B,
                         // lambda1, lambda2, beta, n, c, d, h, R, D
    int filter, variant, climb, n;
    int N;               // current image count
    int kind;
    // FIRE state
    double dt, alpha;
    int npos, fresh;
    // outputs of the last step
    double P, FF, VV, fmax;
    double cv, cf;       // velocity mixing of the step
    long long steps;     // FIRE moves taken
    long long move_limit;// no move once steps reaches this
    int ci;              // climbing image (-1: none)
    int converged;       // fmax < ftol at the last evaluation
    int move;            // the last step moved the images
    int status;
    int stale;           // every image rebuilds at the next evaluation
    int tune_rebuild;    // rebuild at every evaluation (autotuning)
    int row_refine;      // bins along the innermost axis per bin width (>= 1)
    int pad_rr;
    // completion counter of band pass 2 (zero between launches; the last
    // block of the band resets it) and the running fmax^2 as the bits of a
    // non-negative double (ordered like the values)
    unsigned int done_b, pad_done;
    unsigned long long fmax2_bits;
    // image-range shard of a band spread over several devices: the end
    // images are neighbours' images (ghosts), the climbing image comes from
    // the caller (ci_ext: local index, or -1 for none in this range) and
    // the FIRE sums of pass 2 are left in P, FF, VV, fmax (squared) for the
    // caller to combine; the FIRE decision then takes the global sums
    int shard, ci_ext;
    TP<float> tpf;       // Tersoff constants in FP32 / FP64 (Tersoff bands)
    TP<double> tpd;
};

template <typename T> __host__ __device__ inline const TP<T> &tp_of(const BandParams &p);
template <> __host__ __device__ inline const TP<float> &tp_of<float>(const BandParams &p) {
    return p.tpf;
}
template <> __host__ __device__ inline const TP<double> &tp_of<double>(const BandParams &p) {
    return p.tpd;
}

// A bin's three indices in one int, 10 bits each (bin_grid keeps nb_a <=
// 1024): the kernels that walk a slot's stencil unpack them with shifts
// instead of dividing the linear index by the grid's extents.
__host__ __device__ inline int pack_bin(int b0, int b1, int b2) {
    return b0 | (b1 << 10) | (b2 << 20);
}
__host__ __device__ inline void unpack_bin(int p, int &b0, int &b1, int &b2) {
    b0 = p & 1023;
    b1 = (p >> 10) & 1023;
    b2 = p >> 20;
}

struct BandDev {
    int n, rows, ncap, nbins_cap;
    int atpi, rtpi;      // atom tiles / row tiles per image
    void *X, *F, *Fneb, *v;
    ImgScalars *sc;
    BandParams *bp;
    // cell list (image-major)
    int *bin_count;      // [ncap][nbins_cap]
    int *bin_start;      // [ncap][nbins_cap + 1]
    int *bin_tsum;       // [ncap][tsum_cap] scan tile sums / prefixes
    int tsum_cap;
    int *atom_bin, *atom_rank, *slot_unsorted, *slot_atom, *slot_bin, *atom_slot;  // [ncap][n]
    // (atom_bin: linear bin index; slot_bin: the bin's three indices packed
    // by pack_bin)
    void *atom_off, *slot_off;   // [ncap][n] x 4 T (x, y, z, pad): offsets, leading part
    void *atom_off_lo, *slot_off_lo;  // [ncap][n] x 4 T: offset - leading part
    // neighbour-list reuse: positions and periodic wraps at the last build
    void *ref_X;         // [ncap][rows][3] T: R~ at the build (the layout of X)
    int *atom_wrap;      // [ncap][n][3]: floor(s) at the build
    float *skin_part;    // [ncap][atpi]: per-row-tile max displacement (rtpi used)
    // per-slot neighbour lists: Tersoff (slot, code) pairs of MAXN_TERSOFF
    // entries, or LJ packed entries of lj_cap (0: the LJ kernel walks the
    // cell list directly)
    int lj_cap;
    int *nbr_cnt;        // [ncap][n]
    int *nbr_slot;       // [ncap][MAXN or lj_cap][n]
    int *nbr_code;       // [ncap][MAXN][n]
    unsigned char *nbr_rev;  // [ncap][MAXN][n]: entry of j's list pointing back (255: none)
    const double *nep_w;     // NEP weights [NEP_NW] in FP64 and FP32 (NEP bands)
    const float *nep_wf;
    void *nbr_P;         // [ncap][MAXN][n] x 4 T: partials (x, y, z, pad)
    // partial sums
    double *atom_part;   // [ncap][atpi][NPART]
    double *row_part;    // [ncap][rtpi][NPART]
    // Cartesian output scratch [ncap][n][3] doubles (get_path)
    double *cart;
};

struct Tile {
    int band, img, t, pad;
};

struct ImgRef {
    int band, img;
};

struct LJParams {
    double eps, sigma, rc, ephi_c;   // ephi_c = phi(rc) if shifted, else 0
};


// ---- small helpers ------------------------------------------------------

__host__ __device__ inline double det3(const double *m) {
    return m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6]) +
           m[2] * (m[3] * m[7] - m[4] * m[6]);
}

__host__ __device__ inline void inv3(const double *m, double *o) {
    double d = det3(m);
    double id = 1.0 / d;
    o[0] = (m[4] * m[8] - m[5] * m[7]) * id;
    o[1] = (m[2] * m[7] - m[1] * m[8]) * id;
    o[2] = (m[1] * m[5] - m[2] * m[4]) * id;
    o[3] = (m[5] * m[6] - m[3] * m[8]) * id;
    o[4] = (m[0] * m[8] - m[2] * m[6]) * id;
    o[5] = (m[2] * m[3] - m[0] * m[5]) * id;
    o[6] = (m[3] * m[7] - m[4] * m[6]) * id;
    o[7] = (m[1] * m[6] - m[0] * m[7]) * id;
    o[8] = (m[0] * m[4] - m[1] * m[3]) * id;
}

// FP64 reciprocal and reciprocal square root from an FP32 seed and two
// Newton-Raphson steps (relative error ~1e-7 -> ~1e-14 -> ~1 ulp).  FP64
// divide and square root are long instruction sequences on this GPU; these
// serve the per-image 3x3 chains (map-back, list decisions), which run on
// one thread per image.  Arguments must lie within FP32's normal range.
__device__ inline double rcp64(double x) {
    double r = (double)(1.0f / (float)x);
    r = r * (2.0 - x * r);
    r = r * (2.0 - x * r);
    return r;
}
__device__ inline double rsqrt64(double x) {
    double y = (double)rsqrtf((float)x);
    y = y * (1.5 - 0.5 * x * y * y);
    y = y * (1.5 - 0.5 * x * y * y);
    return y;
}
__device__ inline double sqrt64(double x) { return x > 0.0 ? x * rsqrt64(x) : 0.0; }

__host__ __device__ inline void matmul3(const double *a, const double *b, double *o) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            o[3 * i + j] = a[3 * i] * b[j] + a[3 * i + 1] * b[3 + j] + a[3 * i + 2] * b[6 + j];
}

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double4_32a; };

// packed stencil offset: 5 bits per axis, biased by 16
__host__ __device__ inline int pack_code(int d0, int d1, int d2) {
    return (d0 + 16) | ((d1 + 16) << 5) | ((d2 + 16) << 10);
}
__host__ __device__ inline int neg_code(int code) {
    int d0 = (code & 31) - 16, d1 = ((code >> 5) & 31) - 16, d2 = ((code >> 10) & 31) - 16;
    return pack_code(-d0, -d1, -d2);
}

__device__ inline float to_float_ru(float x) { return x; }
__device__ inline float to_float_ru(double x) { return __double2float_ru(x); }

// deterministic warp sum (fixed butterfly)
__device__ inline double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ inline double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ---- lane-parallel 3x3 algebra (map-back, lattice force) -------------------
//
// One warp per image: lane l holds entry (i, j) = (l / 3, l % 3) of each
// 3x3 matrix (lanes 9..31 mirror lane l % 9; their results are unused).  A
// product is then 6 shuffles and a chain of 3 FP64 operations per lane
// instead of 27 dependent-heavy operations in one thread: the map-back is on
// the critical path of every step and FP64 latency (~64 cycles) dominates it.
struct Lane3 {
    int l, i, j;
    __device__ Lane3() : l((int)(threadIdx.x & 31) % 9), i(l / 3), j(l % 3) {}
    __device__ double eye() const { return i == j ? 1.0 : 0.0; }
};
__device__ inline double lget(double a, int src) { return __shfl_sync(0xffffffffu, a, src); }
// (A B)_ij = sum_k A_ik B_kj
__device__ inline double lmul(double a, double b, const Lane3 &p) {
    const double a0 = lget(a, 3 * p.i), a1 = lget(a, 3 * p.i + 1), a2 = lget(a, 3 * p.i + 2);
    const double b0 = lget(b, p.j), b1 = lget(b, 3 + p.j), b2 = lget(b, 6 + p.j);
    return fma(a2, b2, fma(a1, b1, a0 * b0));
}
__device__ inline double ltrans(double a, const Lane3 &p) { return lget(a, 3 * p.j + p.i); }
// cofactor C_ij = A_{i+1,j+1} A_{i+2,j+2} - A_{i+1,j+2} A_{i+2,j+1}
__device__ inline double lcof(double a, const Lane3 &p) {
    const int i1 = (p.i + 1) % 3, i2 = (p.i + 2) % 3, j1 = (p.j + 1) % 3, j2 = (p.j + 2) % 3;
    const double p11 = lget(a, 3 * i1 + j1), p22 = lget(a, 3 * i2 + j2);
    const double p12 = lget(a, 3 * i1 + j2), p21 = lget(a, 3 * i2 + j1);
    return fma(p11, p22, -(p12 * p21));
}
// det A = sum_j A_0j C_0j, in every lane
__device__ inline double ldet(double a, double c) {
    const double t = a * c;
    return lget(t, 0) + lget(t, 1) + lget(t, 2);
}

// The cell of an image from its lattice rows (Sec. II.C), one warp: lane l
// passes entry (l % 9) / 3, (l % 9) % 3 of X_lat (lanes 9..31 mirror, as
// for every lane-parallel 3x3 below).  B = X_lat / c and D = B^(1/2), the
// symmetric root, by the coupled Newton-Schulz iteration (Y -> B^(1/2),
// Z -> B^(-1/2), B scaled into the iteration's convergence region first),
// for the rotation-free filter; D = X_lat / c for the deformation gradient;
// D = I with the filter off.  Then h = h0 D, h^-1 = D^-1 h0^-1 and
// Omega = |det h|, written with D and D^-1 and their FP32 pairs into sc
// (lanes 0..8; Omega by lane 0).  Returns false, with D = I, when B (or the
// deformation gradient) is not positive definite.
// The band constants the cell needs, as one lane's share (entry l = lane %
// 9 of h0 and h0^-1): loaded together, ahead of the FP64 work.
struct CellIn {
    int filter, variant;
    double c, h0, h0inv;
};
__device__ inline CellIn cell_in(const BandParams *bp) {
    const int l = (int)(threadIdx.x & 31) % 9;
    return {bp->filter, bp->variant, bp->c, bp->h0[l], bp->h0inv[l]};
}

__device__ inline bool image_cell_warp(const CellIn &k, double xlat, ImgScalars &sc,
                                       double &h_out) {
    const Lane3 p;
    const int lane = threadIdx.x & 31;
    double D = p.eye(), Di = p.eye();
    bool ok = true;
    if (k.filter) {
        // lattice rows are stored as c (B - I) (or c (D - I)): B = X / c + I
        const double L = xlat * rcp64(k.c) + p.eye();
        if (k.variant == 0) {
            const double B = 0.5 * (L + ltrans(L, p));
            const double C = lcof(B, p);
            const double det = ldet(B, C);
            // Sylvester's criterion: B00 > 0, the leading 2x2 minor (= C22) > 0, det > 0
            ok = lget(B, 0) > 0.0 && lget(C, 8) > 0.0 && det > 0.0;
            if (ok) {
                // spectrum bracket [det / g^2, g], g = largest Gershgorin row bound
                const double rs = fabs(lget(B, 3 * p.i)) + fabs(lget(B, 3 * p.i + 1)) +
                                  fabs(lget(B, 3 * p.i + 2));
                const double g = fmax(fmax(lget(rs, 0), lget(rs, 3)), lget(rs, 6));
                const double ig = rcp64(g);
                const double mu = 0.5 * (g + det * ig * ig);
                double Y = B * rcp64(mu), Z = p.eye();
                for (int it = 0; it < 40; ++it) {
                    const double e = p.eye() - lmul(Z, Y, p);  // I - Z Y
                    const double Tm = p.eye() + 0.5 * e;       // (3I - Z Y) / 2
                    float dev = fabsf((float)e);
                    for (int o = 16; o > 0; o >>= 1)
                        dev = fmaxf(dev, __shfl_xor_sync(0xffffffffu, dev, o));
                    const double Y1 = lmul(Y, Tm, p), Z1 = lmul(Tm, Z, p);
                    Y = Y1;
                    Z = Z1;
                    if (dev < 1e-9f) break;  // the last step took it to ~1e-18
                }
                const double rmu = sqrt64(mu);
                D = 0.5 * (Y + ltrans(Y, p)) * rmu;
                Di = 0.5 * (Z + ltrans(Z, p)) * rcp64(rmu);
            }
        } else {
            const double C = lcof(L, p);
            const double det = ldet(L, C);
            ok = det > 0.0;
            if (ok) {
                D = L;
                Di = ltrans(C, p) * rcp64(det);
            }
        }
    }
    if (!ok) D = Di = p.eye();
    const double h = lmul(k.h0, D, p);
    const double hinv = lmul(Di, k.h0inv, p);  // (h0 D)^-1 = D^-1 h0^-1
    const double omega = fabs(ldet(h, lcof(h, p)));
    if (lane < 9) {
        sc.D[lane] = D;
        sc.Dinv[lane] = Di;
        sc.h[lane] = h;
        sc.hinv[lane] = hinv;
        // FP32 pairs of D and h and FP32 h0^-1 for the FP32 cell-list path
        const float Dh = (float)D, hh = (float)h;
        sc.dfl[lane] = Dh;
        sc.dfl[9 + lane] = (float)(D - (double)Dh);
        sc.dfl[18 + lane] = hh;
        sc.dfl[27 + lane] = (float)(h - (double)hh);
        sc.dfl[36 + lane] = (float)k.h0inv;
    }
    if (lane == 0) sc.omega = omega;
    h_out = h;
    return ok;
}

// Bin vectors of the image's grid for its current cell, one entry per lane
// (lanes 0..8; the whole warp calls): bv_a on a grid of q = 2^(e - 19),
// 2^e >= max |h_a / nb_a|, so every sum of three products delta_a bv_a
// (|delta| <= 7) is exact in FP32; dh = h - nb bv carries the (sub-1e-4 A)
// quantisation to the periodic wrap.  Only the binade of max |h_a / nb_a|
// matters; found in FP32 it can be one binade low by an ulp, and then
// |bv| <= (2^19 + 1) q: three terms |delta| <= 7 still sum below 2^24 q.
// nba = sc.nb[(lane % 9) / 3] and h = sc.h[lane % 9] are passed in (lanes
// 9..31 mirror lane % 9; only lanes 0..8 store).
__device__ inline void bin_vectors_warp(ImgScalars &sc, int nba, double h) {
    const int lane = threadIdx.x & 31;
    const int l = lane % 9;
    float bmax = fabsf((float)h / (float)nba);
    for (int o = 16; o > 0; o >>= 1) bmax = fmaxf(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
    const int e = ilogbf(bmax) + 1 - 19;
    const double q = ldexp(1.0, e), iq = ldexp(1.0, -e);  // exact powers of two
    const double v = q * rint(h * rcp64((double)nba) * iq);
    if (lane < 9) {
        sc.bv[l] = v;
        sc.bvf[l] = (float)v;
        sc.dh[l] = h - nba * v;
        sc.dhf[l] = (float)(h - nba * v);
    }
}

// upper bound of the spectral norm of a 3x3 matrix: the smaller of the
// Frobenius norm and sqrt(|A|_1 |A|_inf), in FP32 and raised by 1e-6 to
// stay a bound
__device__ inline float norm2_bound(const float *A) {
    float f = 0.0f, c1 = 0.0f, ci = 0.0f;
    for (int i = 0; i < 3; ++i) {
        float rs = 0.0f, cs = 0.0f;
        for (int j = 0; j < 3; ++j) {
            f += A[3 * i + j] * A[3 * i + j];
            rs += fabsf(A[3 * i + j]);
            cs += fabsf(A[3 * j + i]);
        }
        ci = fmaxf(ci, rs);
        c1 = fmaxf(c1, cs);
    }
    return fminf(sqrtf(f), sqrtf(c1 * ci)) * 1.000001f;
}

// FP32 inverse of a 3x3 matrix (cofactors over the determinant)
__device__ inline void inv3f(const float *m, float *o) {
    const float c00 = m[4] * m[8] - m[5] * m[7], c01 = m[5] * m[6] - m[3] * m[8],
                c02 = m[3] * m[7] - m[4] * m[6];
    const float id = 1.0f / (m[0] * c00 + m[1] * c01 + m[2] * c02);
    o[0] = c00 * id;
    o[1] = (m[2] * m[7] - m[1] * m[8]) * id;
    o[2] = (m[1] * m[5] - m[2] * m[4]) * id;
    o[3] = c01 * id;
    o[4] = (m[0] * m[8] - m[2] * m[6]) * id;
    o[5] = (m[2] * m[3] - m[0] * m[5]) * id;
    o[6] = c02 * id;
    o[7] = (m[1] * m[6] - m[0] * m[7]) * id;
    o[8] = (m[0] * m[4] - m[1] * m[3]) * id;
}

// The cell's part of the list-reuse bound (one thread): with M = D_b^-1 D - I
// (D_b = D at the build), skin_e = |M|_2 bound and skin_nD = |D|_2 bound, in
// FP32: M - I is small, so its FP32 rounding (~1e-7 absolute) moves the
// bound by far less than the 1e-5 margins, which also cover the FP32 list
// test and displacement.  D from its FP32 leading part, D_b^-1 from the
// build (Dbi: sc.Dbif, or a copy of it loaded ahead).
__device__ inline void skin_terms(ImgScalars &sc, const float *Dbi) {
    const float *D = sc.dfl;
    float M[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            M[3 * i + j] = Dbi[3 * i] * D[j] + Dbi[3 * i + 1] * D[3 + j] +
                           Dbi[3 * i + 2] * D[6 + j] - (i == j ? 1.0f : 0.0f);
    sc.skin_e = norm2_bound(M) * 1.00001f + 1e-6f;
    sc.skin_nD = norm2_bound(D);
}

// FP64 sums of K values over `count` records (value k of record q at
// rec[q * stride + k]) in a fixed order that needs few FP64 instructions (an
// FP64 instruction occupies a warp's FP64 pipe for ~64 cycles here, so
// butterflies over many warps cost more than the sums themselves): thread
// k + K g (g < G) adds value k of records g, g + G, g + 2G, ... in turn, and
// thread k (< K) then adds the G partial sums in order and returns total k.
// Needs blockDim.x >= K G; every thread of the block must call it.
template <int K, int G>
__device__ inline double block_sum_records(const double *rec, int stride, int count) {
    __shared__ double s_part[G * K];
    const int tid = threadIdx.x;
    if (tid < K * G) {
        // four interleaved accumulators (records g, g + G, g + 2G, g + 3G go
        // to accumulators 0..3 in turn): a quarter of the dependent FP64 add
        // chain, with the loads of each round in flight together
        const int k = tid % K, g = tid / K;
        double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
        int q = g;
        for (; q + 3 * G < count; q += 4 * G) {
            v0 += rec[(size_t)q * stride + k];
            v1 += rec[(size_t)(q + G) * stride + k];
            v2 += rec[(size_t)(q + 2 * G) * stride + k];
            v3 += rec[(size_t)(q + 3 * G) * stride + k];
        }
        if (q < count) v0 += rec[(size_t)q * stride + k];
        if (q + G < count) v1 += rec[(size_t)(q + G) * stride + k];
        if (q + 2 * G < count) v2 += rec[(size_t)(q + 2 * G) * stride + k];
        s_part[g * K + k] = (v0 + v1) + (v2 + v3);
    }
    __syncthreads();
    double tot = 0.0;
    if (tid < K)
        for (int g = 0; g < G; ++g) tot += s_part[g * K + tid];
    __syncthreads();
    return tot;
}

// FP64 sums of K values over `count` records like block_sum_records, with
// the loads in flight together: thread k + K g (g < G = NT / K) loads value
// k of records g, g + G, ..., g + (U - 1) G at once and adds them in that
// order (U G records per round trip instead of a chain of four), then the
// G partial sums are added in H = 8 strided groups and the groups in
// order.  The FP64 add count is the same; the round trips fall from
// count / 4G to count / UG.  CG: loads bypass L1 (records written by other
// blocks of the running kernel).  NT = blockDim.x; every thread calls.
template <int K, int U, int NT, bool CG>
__device__ inline double block_sum_records_wide(const double *rec, int stride, int count) {
    constexpr int G = NT / K, H = 8;
    static_assert(G >= H, "too few threads for the group sums");
    __shared__ double s_part[G * K];
    __shared__ double s_grp[H * K];
    const int tid = threadIdx.x;
    if (tid < K * G) {
        const int k = tid % K, g = tid / K;
        double v = 0.0;
        for (int q0 = g; q0 < count; q0 += U * G) {
            double w[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int q = q0 + u * G;
                const double *p = rec + (size_t)q * stride + k;
                w[u] = q < count ? (CG ? __ldcg(p) : *p) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) v += w[u];
        }
        s_part[g * K + k] = v;
    }
    __syncthreads();
    if (tid < K * H) {
        const int k = tid % K, h = tid / K;
        double v = 0.0;
        for (int g = h; g < G; g += H) v += s_part[g * K + k];
        s_grp[h * K + k] = v;
    }
    __syncthreads();
    double tot = 0.0;
    if (tid < K)
        for (int h = 0; h < H; ++h) tot += s_grp[h * K + tid];
    __syncthreads();
    return tot;
}

// Sum K per-thread values over a TILE-thread block in FP64 (fixed order);
// thread 0 of the block receives the totals in out[0..K-1].
template <int K>
__device__ inline void block_sum(double (&v)[K], double *out) {
    __shared__ double red[TILE / 32][K > 0 ? K : 1];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double s = warp_sum(v[k]);
        if (lane == 0) red[w][k] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double s = 0.0;
            for (int q = 0; q < TILE / 32; ++q) s += red[q][k];
            out[k] = s;
        }
    }
    __syncthreads();  // red[] may be reused by a later call
}

// Sum K per-thread values of type T over a TILE-thread block: within each
// warp in T (fixed butterfly), across warps in FP64; thread 0 receives the
// totals.  With T = float the long accumulations (across warps, tiles and
// images) stay FP64 while the per-element work avoids FP64 arithmetic.
template <int K, typename T>
__device__ inline void block_sum_t(T (&v)[K], double *out) {
    __shared__ double red[TILE / 32][K > 0 ? K : 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        T s = v[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[w][k] = (double)s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double s = 0.0;
            for (int q = 0; q < TILE / 32; ++q) s += red[q][k];
            out[k] = s;
        }
    }
    __syncthreads();
}

// As block_sum_t, but the totals go straight to dst[0..K-1]: lane k of warp
// 0 sums value k across the warps, in the same order (so the same bits), and
// the FP64 additions take K/32 warp instructions instead of K in thread 0
// (an FP64 instruction occupies a warp's FP64 pipe for ~64 cycles here).
template <int K, typename T>
__device__ inline void block_sum_store(T (&v)[K], double *dst) {
    static_assert(K <= 32, "one lane per value");
    __shared__ T red[TILE / 32][K > 0 ? K : 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        T s = v[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[w][k] = s;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double s = 0.0;
        for (int q = 0; q < TILE / 32; ++q) s += (double)red[q][threadIdx.x];
        dst[threadIdx.x] = s;
    }
    __syncthreads();
}

// As block_sum_store for K <= 16 values, with a transposing warp reduction:
// at each butterfly level a lane keeps half of its values and adds the
// partner's copy of that half (16 shuffles in all instead of 5 per value),
// so lane l ends with the warp total of value l >> 1.  Fixed order; the
// totals go to dst[0..K-1] in FP64 (across the warps, in warp order).
template <int K, typename T>
__device__ inline void block_sum_store_tr(const T (&v)[K], double *dst) {
    static_assert(K <= 16, "values are padded to 16");
    __shared__ T red[TILE / 32][16];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T a[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = k < K ? v[k] : (T)0;
#pragma unroll
    for (int h = 8, o = 16; h >= 1; h >>= 1, o >>= 1) {
        const bool hi = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < h; ++k) {
            const T send = hi ? a[k] : a[k + h];
            const T keep = hi ? a[k + h] : a[k];
            a[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    a[0] += __shfl_xor_sync(0xffffffffu, a[0], 1);
    if ((lane & 1) == 0) red[w][lane >> 1] = a[0];
    __syncthreads();
    if (threadIdx.x < K) {
        double s = 0.0;
        for (int q = 0; q < TILE / 32; ++q) s += (double)red[q][threadIdx.x];
        dst[threadIdx.x] = s;
    }
    __syncthreads();
}

// Sum K per-thread values over a block of any multiple of 32 threads (up to
// 1024) in FP64, fixed order (a warp butterfly within each warp, then one
// across the warp totals); thread 0 receives the totals.  Butterflies keep
// the dependent FP64 chain at 5 + 5 additions (a dependent FP64 operation
// costs ~64 cycles here).
template <int K>
__device__ inline void block_sum_any(double (&v)[K], double *out) {
    __shared__ double red[32][K];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const double s = warp_sum(v[k]);
        if (lane == 0) red[w][k] = s;
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const double s = warp_sum(lane < nw ? red[lane][k] : 0.0);
            if (lane == 0) out[k] = s;
        }
    }
    __syncthreads();
}

// block-wide maximum; thread 0 receives it
__device__ inline double block_max_any(double v) {
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_max(v);
    if (lane == 0) red[w] = v;
    __syncthreads();
    double m = red[0];
    if (threadIdx.x == 0)
        for (int q = 1; q < nw; ++q) m = fmax(m, red[q]);
    __syncthreads();
    return m;
}

// threads of the per-image / per-band reduction kernels
constexpr int RED_THREADS = 256;
// threads of the per-image finalize (one block per image: wide record sums)
constexpr int FIN_THREADS = 1024;

// Copy a record between global and shared memory with all threads of the
// block (8-byte words).  The per-image and per-band kernels read many fields
// of ImgScalars and BandParams on one thread; staged first, those reads cost
// one round trip instead of a chain of dependent global loads.
template <typename S>
__device__ inline void stage_copy(S *dst, const S *src) {
    static_assert(sizeof(S) % 8 == 0, "record size must be a multiple of 8 bytes");
    static_assert(alignof(S) >= 8, "record must be 8-byte aligned for word copies");
    // every word loaded before the first store (the compiler cannot tell
    // the shared side from the global one, so interleaved copies would wait
    // out one round trip per word); PER words per thread cover the record
    // for any block of at least 32 threads
    constexpr int NW = (int)(sizeof(S) / 8), PER = (NW + 31) / 32;
    const unsigned long long *s = (const unsigned long long *)src;
    unsigned long long *d = (unsigned long long *)dst;
    unsigned long long w[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = threadIdx.x + k * blockDim.x;
        w[k] = i < NW ? s[i] : 0ull;
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = threadIdx.x + k * blockDim.x;
        if (i < NW) d[i] = w[k];
    }
}

// ---- launchers (defined in the kernel translation units) ---------------

// map-back and the cell-list decision of every image (the displacements
// since the last build come from the last move, per row tile)
template <typename T>
void launch_mapback(const ImgRef *imgs, int count, BandDev *bands, int force, cudaStream_t s);
// bins or offsets; with has_cond also sets `cond` (a conditional graph
// node's handle, default 0) to 1 when a listed image rebuilds its cell list
template <typename T>
void launch_bin_assign(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s,
                       cudaGraphConditionalHandle cond = 0, int has_cond = 0);
// part 0: tile sums, 1: scan of the tile sums, 2: final per-bin scan
void launch_bin_scan(const ImgRef *imgs, int count, int max_bins, BandDev *bands,
                     cudaStream_t s, int part);
void launch_bin_scatter(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s);
template <typename T>
void launch_bin_order(const ImgRef *imgs, int count, int max_bins, BandDev *bands,
                      cudaStream_t s);
template <typename T>
void launch_lj(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s);
template <typename T>
void launch_lj_list(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s);
// minb: resident blocks per SM of the force kernel variant (FP32: 5-8 for
// LJ, 4-8 for Tersoff; the autotuner picks it)
template <typename T>
void launch_lj_nbr(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s, int minb);
template <typename T>
void launch_tersoff_list(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s);
template <typename T>
void launch_tersoff_reverse(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s);
template <typename T>
void launch_tersoff_partials(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s,
                             int minb);
template <typename T>
void launch_nep_partials(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s);
template <typename T>
void launch_tersoff_gather(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s);
template <typename T>
void launch_image_finalize(const ImgRef *imgs, int count, BandDev *bands, cudaStream_t s);
// band pass 1 (dots, then per image and per band the NEB coefficients and
// FIRE sums), pass 2 (f_NEB, fmax, FIRE decision); the dots alone and their
// per-image sums (spacings of the refinement check)
template <typename T>
void launch_band_dots(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s);
template <typename T>
void launch_neb_force(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s);
template <typename T>
void launch_band_dots_only(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s);
void launch_dots_reduce(const ImgRef *imgs, int count, BandDev *bands, cudaStream_t s);
// the FIRE decision of a shard on the global sums (P, F.F, v.v, fmax^2)
void launch_shard_fire(BandDev *band, double P, double FF, double VV, double fmax2,
                       cudaStream_t s);
template <typename T>
void launch_fire_update(const Tile *tiles, int ntiles, const ImgRef *imgs, int nimg,
                        BandDev *bands, cudaStream_t s);
template <typename T>
void launch_energy64(const Tile *tiles, int ntiles, const ImgRef *imgs, int nimg, BandDev *bands,
                     cudaStream_t s);
template <typename T>
void launch_cartesian(const ImgRef *imgs, int count, int max_n, BandDev *bands, cudaStream_t s);
template <typename T>
void launch_midpoint(BandDev *band, int img, int rows, cudaStream_t s);
void launch_gather_status(BandDev *bands, int nb, double *out, cudaStream_t s);
template <typename T>
void launch_setup(const double *R0, const double *R1, const double *noise, int n, int N,
                  BandDev *band, cudaStream_t s, const double *h1);

}  // namespace cfneb
