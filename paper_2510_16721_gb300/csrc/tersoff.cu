// Tersoff (1988 form, lambda3 = 0) energy, forces and virial.
//
//   U_i = 1/2 sum_j fC(r_ij) [A e^{-l1 r_ij} - b_ij B e^{-l2 r_ij}]
//   b_ij = (1 + (beta zeta_ij)^n)^(-1/2n),
//   zeta_ij = sum_{k != j} fC(r_ik) g(cos theta_ijk)
//
// Two kernels, both one thread per atom in cell-list slot order:
//
// 1. k_ters_partials: collects the neighbour entries (j, periodic shift)
//    of atom i inside R + D from the cell list, and computes the site energy
//    U_i and every partial P_ij = dU_i/dr^ij (Sec. II.B, Eq. U: U_i is a
//    function of the r^ij of i's neighbours).  It also accumulates the
//    virial in its per-site form V_mn = -sum_i sum_j P_ij,n r^ij_m (first
//    line of the derivation of Eq. V2), which needs no pair forces.
// 2. k_ters_gather: F_i = sum_j f^ij with f^ij = P_ij - P_ji (Sec. II.B),
//    where P_ji is read from j's list at the entry that points back to i
//    under the opposite shift.  No atomics: each atom sums its own terms in
//    list order, so the result is deterministic.
//
// The angular function is evaluated as g = 1 + c^2 u^2 / (d^2 (d^2 + u^2)),
// u = h - cos theta: algebraically Tersoff's 1 + c^2/d^2 - c^2/(d^2 + u^2),
// but free of the cancellation between two ~8e7 terms that would cost FP32
// four digits.
//
// Distances are carried to twice the working precision.  With n < 1 the
// bond-order derivative grows like zeta^(n-1) when a neighbour nears R + D,
// so forces there respond to a distance error d like d^0.46: ~1e-4 eV/A for
// the 1e-7 A that an FP32 pair vector near 2 A can hold.  Each atom's
// offset is stored as a leading FP32 part on a 2^-20 A grid plus the FP32
// remainder; a pair vector's leading part (o_j - o_i) + c is then exact in
// plain FP32 (c, the displacement between bin centres, lies on a coarser
// power-of-two grid by construction), its low part collects the remainders
// and the periodic-wrap correction, and s = r - R follows from r^2 - R^2
// with FMA-exact squares.  (FP64 bands use Knuth's two-sum instead.)  Directions and angles use the leading part; every radial
// function (f_C, f_R, f_A and derivatives) uses s, accurate to ~1e-12 A.
// exp(-l r) is evaluated as exp(-l R) exp(-l s).  The cutoff function is
// written without cancellation: with a = pi (D - s) / 4D and
// b = pi (D + s) / 4D (a + b = pi/2), 1/2 - 1/2 sin(pi s / 2D) = sin^2 a and
// its derivative -(pi/4D) cos(pi s / 2D) = -(pi/2D) sin a sin b; D - s and
// D + s are formed exactly (two-term D), so f_C keeps full relative accuracy
// even where it is 1e-8 (a neighbour at the outer edge, where the bond-order
// derivative amplifies any absolute error).
#include "common.cuh"

namespace cfneb {

template <typename T> struct M;
template <> struct M<float> {
    static __device__ float ex(float x) { return expf(x); }
    static __device__ float lg(float x) { return logf(x); }
    static __device__ float l1p(float x) { return log1pf(x); }
    static __device__ float sq(float x) { return sqrtf(x); }
    static __device__ float sn(float x) { return sinf(x); }
    // correctly rounded reciprocal: a short sequence, unlike a full divide
    static __device__ float rcp(float x) { return __frcp_rn(x); }
    // the fast division intrinsic (2 ulp) where only relative accuracy of a
    // factor matters (1/r of directions, the angular function)
    static __device__ float rcpf(float x) { return __fdividef(1.0f, x); }
};
template <> struct M<double> {
    static __device__ double ex(double x) { return exp(x); }
    static __device__ double lg(double x) { return log(x); }
    static __device__ double l1p(double x) { return log1p(x); }
    static __device__ double sq(double x) { return sqrt(x); }
    static __device__ double sn(double x) { return sin(x); }
    static __device__ double rcp(double x) { return 1.0 / x; }
    static __device__ double rcpf(double x) { return 1.0 / x; }
};

__device__ inline float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ inline double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ inline float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ inline double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ inline float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ inline double sub_rn(double a, double b) { return __dsub_rn(a, b); }

// Knuth's two-sum: s + e == a + b exactly
template <typename T>
__device__ inline void two_sum(T a, T b, T &s, T &e) {
    s = add_rn(a, b);
    const T bb = sub_rn(s, a);
    e = add_rn(sub_rn(a, sub_rn(s, bb)), sub_rn(b, bb));
}

// Dekker's fast two-sum (|a| >= |b|): s + e == a + b exactly
template <typename T>
__device__ inline void fast_two_sum(T a, T b, T &s, T &e) {
    s = add_rn(a, b);
    e = sub_rn(b, sub_rn(s, a));
}

// r and s = r - R for the pair vector (x + xl, y + yl, z + zl), leading
// parts x, y, z and small remainders xl, yl, zl
template <typename T>
__device__ inline void dist_s(const TP<T> &q, T x, T y, T z, T xl, T yl, T zl, T &r, T &s) {
    const T px = mul_rn(x, x), py = mul_rn(y, y), pz = mul_rn(z, z);
    const T ex = fma(x, x, -px) + (T)2 * x * xl, ey = fma(y, y, -py) + (T)2 * y * yl,
            ez = fma(z, z, -pz) + (T)2 * z * zl;
    T s1, e1, s2, e2;
    two_sum(px, py, s1, e1);
    two_sum(s1, pz, s2, e2);
    const T lo = add_rn(add_rn(add_rn(ex, ey), ez), add_rn(e1, e2));
    // s2 - R^2 is exact when r^2 lies within a factor 2 of R^2
    const T d = add_rn(sub_rn(s2, q.R2hi), sub_rn(lo, q.R2lo));
    r = M<T>::sq(add_rn(s2, lo));
    s = d * M<T>::rcp(r + q.R);
}

// sin a for a in [0, pi/2], the cutoff's only arguments.  FP32: the Taylor
// series to the a^13 term in nested form, sin a = a (1 - a^2/(2.3) (1 -
// a^2/(4.5) (1 - ...))) (truncation below 7e-10 relative at pi/2, rounding a
// few ulp, full relative accuracy as a -> 0); a handful of FMAs instead of
// a general-range sine.  FP64: the library sine.
__device__ inline float sin_quarter(float a) {
    const float a2 = a * a;
    float p = 1.0f - a2 * (1.0f / 156.0f);
    p = 1.0f - a2 * (1.0f / 110.0f) * p;
    p = 1.0f - a2 * (1.0f / 72.0f) * p;
    p = 1.0f - a2 * (1.0f / 42.0f) * p;
    p = 1.0f - a2 * (1.0f / 20.0f) * p;
    p = 1.0f - a2 * (1.0f / 6.0f) * p;
    return a * p;
}
__device__ inline double sin_quarter(double a) { return sin(a); }

// cutoff function and derivative from s = r - R (see the header comment)
template <typename T>
__device__ inline void cutoff(const TP<T> &q, T s, T &fc, T &dfc) {
    const T u = sub_rn(q.D, s) + q.Dlo;  // D - s
    const T v = add_rn(q.D, s) + q.Dlo;  // D + s
    if (v <= (T)0) { fc = (T)1; dfc = (T)0; return; }
    if (u <= (T)0) { fc = (T)0; dfc = (T)0; return; }
    const T sa = sin_quarter(q.pi_4D * u), sb = sin_quarter(q.pi_4D * v);
    fc = sa * sa;
    dfc = -q.pi_2D * sa * sb;
}

// g = 1 + (c^2/d^2) u^2 / (d^2 + u^2) and dg/dcos = -2 c^2 u / (d^2 + u^2)^2
// with u = h - cos, from one reciprocal
template <typename T>
__device__ inline void gfun(const TP<T> &q, T cs, T &g, T &dg) {
    const T u = q.h - cs;
    const T inv = M<T>::rcpf(q.d2 + u * u);
    g = (T)1 + q.c2d2 * u * u * inv;
    dg = -(T)2 * q.c2 * u * inv * inv;
}

// list entries of an atom held in shared memory by the force kernel (atoms
// with more entries keep theirs in local memory)
template <typename T> struct NShared;
template <> struct NShared<float> { static constexpr int value = 6; };
template <> struct NShared<double> { static constexpr int value = 4; };

// Per-thread neighbour records: field f of entry k at p[(f * cap + k) * stride]
// (stride TILE in shared memory, 1 in a local array).
enum { NB_RX, NB_RY, NB_RZ, NB_SR, NB_IR, NB_FC, NB_DFC, NB_PX, NB_PY, NB_PZ, NB_FIELDS };
template <typename T>
struct Nbr {
    T *p;
    int stride, cap;
    __device__ T &operator()(int f, int k) const { return p[(f * cap + k) * stride]; }
};

// Pair vector of entry (slot qs, stencil code) of slot t: leading parts
// x, y, z (directions) and s = r - R to twice the working precision.
// (b0, b1, b2) is t's bin; the entry's bin offset and periodic wrap follow
// from the code.
template <typename T>
__device__ inline void ters_pair(const TP<T> &q, const typename Vec4<T>::type &oi,
                                 const typename Vec4<T>::type &oil,
                                 const typename Vec4<T>::type &oj,
                                 const typename Vec4<T>::type &ojl, int code, int b0, int b1,
                                 int b2, const T *s_bv, const T *s_dh, const int *s_nb, T &x,
                                 T &y, T &z, T &s) {
    const int d0 = (code & 31) - 16, d1 = ((code >> 5) & 31) - 16, d2 = ((code >> 10) & 31) - 16;
    int w0 = b0 + d0, t0 = 0, w1 = b1 + d1, t1 = 0, w2 = b2 + d2, t2 = 0;
    while (w0 < 0) { w0 += s_nb[0]; --t0; }
    while (w0 >= s_nb[0]) { w0 -= s_nb[0]; ++t0; }
    while (w1 < 0) { w1 += s_nb[1]; --t1; }
    while (w1 >= s_nb[1]) { w1 -= s_nb[1]; ++t1; }
    while (w2 < 0) { w2 += s_nb[2]; --t2; }
    while (w2 >= s_nb[2]) { w2 -= s_nb[2]; ++t2; }
    // bin-centre displacement: exact (quantised bin vectors)
    const T cx = d0 * s_bv[0] + d1 * s_bv[3] + d2 * s_bv[6];
    const T cy = d0 * s_bv[1] + d1 * s_bv[4] + d2 * s_bv[7];
    const T cz = d0 * s_bv[2] + d1 * s_bv[5] + d2 * s_bv[8];
    // periodic-wrap remainder (tiny)
    const T wx = t0 * s_dh[0] + t1 * s_dh[3] + t2 * s_dh[6];
    const T wy = t0 * s_dh[1] + t1 * s_dh[4] + t2 * s_dh[7];
    const T wz = t0 * s_dh[2] + t1 * s_dh[5] + t2 * s_dh[8];
    T xl, yl, zl;
    if (sizeof(T) == 4) {
        // FP32 offsets of many-body bands lie on a 2^-20 A grid (the offset
        // refresh rounds them there): (o_j - o_i) + c is exact as it stands
        x = add_rn(sub_rn(oj.x, oi.x), cx);
        y = add_rn(sub_rn(oj.y, oi.y), cy);
        z = add_rn(sub_rn(oj.z, oi.z), cz);
        xl = add_rn(sub_rn(ojl.x, oil.x), wx);
        yl = add_rn(sub_rn(ojl.y, oil.y), wy);
        zl = add_rn(sub_rn(ojl.z, oil.z), wz);
    } else {
        T ex1, ey1, ez1, ex2, ey2, ez2;
        two_sum(oj.x, -oi.x, x, ex1);
        two_sum(oj.y, -oi.y, y, ey1);
        two_sum(oj.z, -oi.z, z, ez1);
        two_sum(x, cx, x, ex2);
        two_sum(y, cy, y, ey2);
        two_sum(z, cz, z, ez2);
        xl = ((ojl.x - oil.x) + wx) + (ex1 + ex2);
        yl = ((ojl.y - oil.y) + wy) + (ey1 + ey2);
        zl = ((ojl.z - oil.z) + wz) + (ez1 + ez2);
    }
    // renormalise: the leading part (used for directions) takes the wrap
    // remainder, the low part keeps the rest
    fast_two_sum(x, xl, x, xl);
    fast_two_sum(y, yl, y, yl);
    fast_two_sum(z, zl, z, zl);
    T r;
    dist_s(q, x, y, z, xl, yl, zl, r, s);
}

// Neighbour entries of slot t within rl into the global list (slot, stencil
// code); returns the total count.  A plain FP32 screen with a 1e-5 relative
// margin: an entry just outside R + D costs nothing but a zero term.
template <typename T>
__device__ inline int ters_collect_list(T rl2, const BandDev &b, int img, int t, const T *s_bv,
                                        const T *s_dh, const int *s_nb, const int *s_m) {
    using T4 = typename Vec4<T>::type;
    const int n = b.n;
    const size_t base = (size_t)img * n;
    const T4 *off = (const T4 *)b.slot_off + base;
    const int *start = b.bin_start + (size_t)img * (b.nbins_cap + 1);
    int *nslot = b.nbr_slot + (size_t)img * MAXN_TERSOFF * n;
    int *ncode = b.nbr_code + (size_t)img * MAXN_TERSOFF * n;
    const T rc2_screen = rl2 * (T)1.00001;
    const int nb1 = s_nb[1], nb2 = s_nb[2];
    int b0, b1, b2;
    unpack_bin(b.slot_bin[base + t], b0, b1, b2);
    const T4 oi = off[t];
    int total = 0;
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
                const T ux0 = (d0 * s_bv[0] + d1 * s_bv[3] + d2 * s_bv[6]) +
                              (t0 * s_dh[0] + t1 * s_dh[3] + t2 * s_dh[6]) - oi.x;
                const T uy0 = (d0 * s_bv[1] + d1 * s_bv[4] + d2 * s_bv[7]) +
                              (t0 * s_dh[1] + t1 * s_dh[4] + t2 * s_dh[7]) - oi.y;
                const T uz0 = (d0 * s_bv[2] + d1 * s_bv[5] + d2 * s_bv[8]) +
                              (t0 * s_dh[2] + t1 * s_dh[5] + t2 * s_dh[8]) - oi.z;
                const int q1 = start[w + 1];
                for (int qs = start[w]; qs < q1; ++qs) {
                    const T4 oj = off[qs];
                    const T ux = oj.x + ux0, uy = oj.y + uy0, uz = oj.z + uz0;
                    const T r2 = ux * ux + uy * uy + uz * uz;
                    // r2 == 0: the atom itself at zero shift
                    if (!(r2 < rc2_screen) || (qs == t && d0 == 0 && d1 == 0 && d2 == 0 &&
                                               t0 == 0 && t1 == 0 && t2 == 0))
                        continue;
                    if (total < MAXN_TERSOFF) {
                        nslot[(size_t)total * n + t] = qs;
                        ncode[(size_t)total * n + t] = pack_code(d0, d1, d2);
                    }
                    ++total;
                }
            }
        }
    }
    return total;
}

// Site energy U_i, partials P_ij (written to the list) and the site virial
// of slot t from its cnt neighbour records (r^ij and s = r - R filled in).
//
// cos theta_jk, g and dg/dcos are symmetric in (j, k), so the angular work
// runs over unordered pairs j < k, each evaluated once per pass:
//   pass 1: zeta_j += fC_k g_jk and zeta_k += fC_j g_jk;
//   pass 2, per j: b_ij, the radial term of P_ij and pref_j = 1/2 fC_j f_A,j
//     db_ij/dzeta_ij (zeta parks in the P_x field, pref in the s field);
//   pass 3: with S = dg_jk (pref_j fC_k + pref_k fC_j),
//     P_ij += S dcos/dr^ij + pref_k dfC_j g_jk r^ij / r_ij,
//     P_ik += S dcos/dr^ik + pref_j dfC_k g_jk r^ik / r_ik
//   (the j-as-bond and k-as-bond terms of dU_i together).  A pair with an
// entry beyond R + D (fC = dfC = 0) contributes nothing and is skipped.
template <typename T>
__device__ inline void ters_site(const TP<T> &q, int cnt, const Nbr<T> &nb,
                                 typename Vec4<T>::type *nP, int n, int t, T &U, T (&vir)[9]) {
    for (int j = 0; j < cnt; ++j) {
        T fc, dfc;
        cutoff(q, nb(NB_SR, j), fc, dfc);
        nb(NB_FC, j) = fc;
        nb(NB_DFC, j) = dfc;
        nb(NB_IR, j) = M<T>::rcpf(q.R + nb(NB_SR, j));  // 1 / r
        nb(NB_PX, j) = (T)0;                             // zeta_ij
    }
    // pass 1: zeta
    for (int j = 0; j < cnt; ++j) {
        const T fcj = nb(NB_FC, j);
        if (fcj == (T)0 && nb(NB_DFC, j) == (T)0) continue;
        const T xj = nb(NB_RX, j), yj = nb(NB_RY, j), zj = nb(NB_RZ, j), irj = nb(NB_IR, j);
        T zj_acc = 0;
        for (int k = j + 1; k < cnt; ++k) {
            const T fck = nb(NB_FC, k);
            if (fck == (T)0 && nb(NB_DFC, k) == (T)0) continue;
            const T cs = (xj * nb(NB_RX, k) + yj * nb(NB_RY, k) + zj * nb(NB_RZ, k)) * irj *
                         nb(NB_IR, k);
            T g, dg;
            gfun(q, cs, g, dg);
            zj_acc += fck * g;
            nb(NB_PX, k) += fcj * g;
        }
        nb(NB_PX, j) += zj_acc;
    }
    // pass 2: bond orders, energy, radial terms, prefactors
    for (int j = 0; j < cnt; ++j) {
        const T fcj = nb(NB_FC, j), dfcj = nb(NB_DFC, j);
        const T xj = nb(NB_RX, j), yj = nb(NB_RY, j), zj = nb(NB_RZ, j);
        if (fcj == (T)0 && dfcj == (T)0) {  // beyond R + D: no terms
            nb(NB_SR, j) = (T)0;
            nb(NB_PX, j) = nb(NB_PY, j) = nb(NB_PZ, j) = (T)0;
            continue;
        }
        const T zeta = nb(NB_PX, j), sj_ = nb(NB_SR, j), irj = nb(NB_IR, j);
        T bij = (T)1, dbij = (T)0;
        if (zeta > (T)0) {
            const T x = M<T>::ex(q.n * M<T>::lg(q.beta * zeta));
            bij = M<T>::ex(-q.inv2n * M<T>::l1p(x));
            dbij = (T)(-0.5) * bij * x / (((T)1 + x) * zeta);
        }
        const T fr = q.AeR * M<T>::ex(-q.l1 * sj_);
        const T fa = -q.BeR * M<T>::ex(-q.l2 * sj_);
        const T dfr = -q.l1 * fr, dfa = -q.l2 * fa;
        U += (T)0.5 * fcj * (fr + bij * fa);
        const T radial = (T)0.5 * (dfcj * (fr + bij * fa) + fcj * (dfr + bij * dfa)) * irj;
        nb(NB_SR, j) = (T)0.5 * fcj * fa * dbij;  // pref_j
        nb(NB_PX, j) = radial * xj;
        nb(NB_PY, j) = radial * yj;
        nb(NB_PZ, j) = radial * zj;
    }
    // pass 3: angular terms
    for (int j = 0; j < cnt; ++j) {
        const T fcj = nb(NB_FC, j), dfcj = nb(NB_DFC, j);
        if (fcj == (T)0 && dfcj == (T)0) continue;
        const T xj = nb(NB_RX, j), yj = nb(NB_RY, j), zj = nb(NB_RZ, j);
        const T irj = nb(NB_IR, j), prefj = nb(NB_SR, j);
        T Pxj = 0, Pyj = 0, Pzj = 0;
        for (int k = j + 1; k < cnt; ++k) {
            const T fck = nb(NB_FC, k), dfck = nb(NB_DFC, k);
            if (fck == (T)0 && dfck == (T)0) continue;
            const T prefk = nb(NB_SR, k);
            if (prefj == (T)0 && prefk == (T)0) continue;
            const T xk = nb(NB_RX, k), yk = nb(NB_RY, k), zk = nb(NB_RZ, k);
            const T irk = nb(NB_IR, k);
            const T ijk = irj * irk;
            const T cs = (xj * xk + yj * yk + zj * zk) * ijk;
            T g, dg;
            gfun(q, cs, g, dg);
            // dcos/dr^ij = r^ik/(r_ij r_ik) - cos r^ij/r_ij^2 (and j <-> k)
            const T aj = cs * irj * irj, ak = cs * irk * irk;
            const T S = dg * (prefj * fck + prefk * fcj);
            const T rj = prefk * dfcj * g * irj, rk = prefj * dfck * g * irk;
            Pxj += S * (xk * ijk - aj * xj) + rj * xj;
            Pyj += S * (yk * ijk - aj * yj) + rj * yj;
            Pzj += S * (zk * ijk - aj * zj) + rj * zj;
            nb(NB_PX, k) += S * (xj * ijk - ak * xk) + rk * xk;
            nb(NB_PY, k) += S * (yj * ijk - ak * yk) + rk * yk;
            nb(NB_PZ, k) += S * (zj * ijk - ak * zk) + rk * zk;
        }
        nb(NB_PX, j) += Pxj;
        nb(NB_PY, j) += Pyj;
        nb(NB_PZ, j) += Pzj;
    }
    for (int j = 0; j < cnt; ++j) {
        const T Px = nb(NB_PX, j), Py = nb(NB_PY, j), Pz = nb(NB_PZ, j);
        const T rx = nb(NB_RX, j), ry = nb(NB_RY, j), rz = nb(NB_RZ, j);
        typename Vec4<T>::type pv;
        pv.x = Px;
        pv.y = Py;
        pv.z = Pz;
        pv.w = (T)0;
        nP[(size_t)j * n + t] = pv;  // one vector store; one vector gather later
        // V_mn -= r_m P_n
        vir[0] -= rx * Px; vir[1] -= rx * Py; vir[2] -= rx * Pz;
        vir[3] -= ry * Px; vir[4] -= ry * Py; vir[5] -= ry * Pz;
        vir[6] -= rz * Px; vir[7] -= rz * Py; vir[8] -= rz * Pz;
    }
}


// Neighbour list of a rebuilt image: one light thread per atom walks the
// cell-list stencil (high occupancy hides the chained bin loads) and writes,
// for each entry within rl, the neighbour slot and the stencil code,
// coalesced as [entry][atom].  Images that keep their cell list keep their
// list too.
template <typename T>
__global__ void __launch_bounds__(TILE) k_ters_list(const Tile *tiles, int ntiles, BandDev *bands) {
    __shared__ T s_bv[9], s_dh[9], s_rl2;
    __shared__ int s_nb[3], s_m[3];
    for (int k = blockIdx.x; k < ntiles; k += gridDim.x) {
        const Tile tl = tiles[k];
        BandDev &b = bands[tl.band];
        const ImgScalars &sc = b.sc[tl.img];
        if (!sc.rebuild) continue;  // uniform over the block
        if (threadIdx.x < 9) {
            s_bv[threadIdx.x] = (T)sc.bv[threadIdx.x];
            s_dh[threadIdx.x] = (T)sc.dh[threadIdx.x];
        }
        if (threadIdx.x < 3) {
            s_nb[threadIdx.x] = sc.nb[threadIdx.x];
            s_m[threadIdx.x] = sc.m[threadIdx.x];
        }
        if (threadIdx.x == 0) {  // FP64 work once per block, not per thread
            const double rl = b.bp->rl > 0.0 ? b.bp->rl : b.bp->rc;
            s_rl2 = (T)(rl * rl);
        }
        __syncthreads();
        const int n = b.n;
        const int t = tl.t * TILE + threadIdx.x;
        if (t < n) {
            const int total = ters_collect_list<T>(s_rl2, b, tl.img, t, s_bv, s_dh, s_nb, s_m);
            b.nbr_cnt[(size_t)tl.img * n + t] = total < MAXN_TERSOFF ? total : MAXN_TERSOFF;
            if (total > MAXN_TERSOFF) atomicOr(&b.bp->status, ST_NBR_OVERFLOW);
        }
        __syncthreads();  // the staged geometry is rewritten for the next tile
    }
}

// pair vectors of the list entries of slot t from the current offsets, into
// its neighbour records
template <typename T>
__device__ inline void ters_load(const TP<T> &q, const BandDev &b, int img, int t, int cnt,
                                 const T *s_bv, const T *s_dh, const int *s_nb,
                                 const Nbr<T> &nb) {
    using T4 = typename Vec4<T>::type;
    const int n = b.n;
    const size_t base = (size_t)img * n;
    const T4 *off = (const T4 *)b.slot_off + base;
    const T4 *offl = (const T4 *)b.slot_off_lo + base;
    const int *nslot = b.nbr_slot + (size_t)img * MAXN_TERSOFF * n;
    const int *ncode = b.nbr_code + (size_t)img * MAXN_TERSOFF * n;
    int b0, b1, b2;
    unpack_bin(b.slot_bin[base + t], b0, b1, b2);
    const T4 oi = off[t], oil = offl[t];
    for (int k = 0; k < cnt; ++k) {
        const int qs = nslot[(size_t)k * n + t];
        const int code = ncode[(size_t)k * n + t];
        T x, y, z, sr;
        ters_pair<T>(q, oi, oil, off[qs], offl[qs], code, b0, b1, b2, s_bv, s_dh, s_nb, x, y, z,
                     sr);
        nb(NB_RX, k) = x;
        nb(NB_RY, k) = y;
        nb(NB_RZ, k) = z;
        nb(NB_SR, k) = sr;
    }
}

// ---- register-resident site computation (FP32 path) -------------------------
//
// Carbon atoms hold 3 (graphite) or 4 (diamond) list entries within R + D +
// skin, 5 or more only in compressed intermediates.  For up to RMAX entries
// the records live in registers: every loop below is unrolled over RMAX with
// the entry index known at compile time, and the angular values (cos, g,
// dg/dcos) of each unordered pair are kept from the zeta pass for the force
// pass instead of being evaluated twice.  Atoms with more entries take the
// record path above (ters_site on a local array).  The arithmetic is that of
// ters_site term by term.
constexpr int RMAX = 4;
constexpr int RPAIRS = RMAX * (RMAX - 1) / 2;

template <typename T>
__device__ inline void ters_load_reg(const TP<T> &q, const BandDev &b, int img, int t, int cnt,
                                     const T *s_bv, const T *s_dh, const int *s_nb,
                                     T (&rx)[RMAX], T (&ry)[RMAX], T (&rz)[RMAX],
                                     T (&sr)[RMAX]) {
    using T4 = typename Vec4<T>::type;
    const int n = b.n;
    const size_t base = (size_t)img * n;
    const T4 *off = (const T4 *)b.slot_off + base;
    const T4 *offl = (const T4 *)b.slot_off_lo + base;
    const int *nslot = b.nbr_slot + (size_t)img * MAXN_TERSOFF * n;
    const int *ncode = b.nbr_code + (size_t)img * MAXN_TERSOFF * n;
    int b0, b1, b2;
    unpack_bin(b.slot_bin[base + t], b0, b1, b2);
    const T4 oi = off[t], oil = offl[t];
    int qs[RMAX], code[RMAX];
#pragma unroll
    for (int k = 0; k < RMAX; ++k) {
        qs[k] = k < cnt ? nslot[(size_t)k * n + t] : t;
        code[k] = k < cnt ? ncode[(size_t)k * n + t] : 0;
    }
#pragma unroll
    for (int k = 0; k < RMAX; ++k) {
        if (k < cnt) {
            ters_pair<T>(q, oi, oil, off[qs[k]], offl[qs[k]], code[k], b0, b1, b2, s_bv, s_dh,
                         s_nb, rx[k], ry[k], rz[k], sr[k]);
        } else {
            rx[k] = ry[k] = rz[k] = (T)0;
            sr[k] = q.D + q.D;  // beyond R + D: no terms
        }
    }
}

template <typename T>
__device__ inline void ters_site_reg(const TP<T> &q, const T (&rx)[RMAX], const T (&ry)[RMAX],
                                     const T (&rz)[RMAX], const T (&sr)[RMAX],
                                     typename Vec4<T>::type *nP, int cnt, int n, int t, T &U,
                                     T (&vir)[9]) {
    T fc[RMAX], dfc[RMAX], ir[RMAX], zeta[RMAX];
    bool act[RMAX];
#pragma unroll
    for (int j = 0; j < RMAX; ++j) {
        cutoff(q, sr[j], fc[j], dfc[j]);
        act[j] = !(fc[j] == (T)0 && dfc[j] == (T)0);
        ir[j] = M<T>::rcpf(q.R + sr[j]);
        zeta[j] = (T)0;
    }
    // pass 1: zeta over unordered pairs; cos, g, dg kept per pair
    T pc[RPAIRS], pg[RPAIRS], pdg[RPAIRS];
    {
        int p = 0;
#pragma unroll
        for (int j = 0; j < RMAX; ++j) {
            T zj_acc = 0;
#pragma unroll
            for (int k = j + 1; k < RMAX; ++k, ++p) {
                pc[p] = pg[p] = pdg[p] = (T)0;
                if (act[j] && act[k]) {
                    const T cs = (rx[j] * rx[k] + ry[j] * ry[k] + rz[j] * rz[k]) * ir[j] * ir[k];
                    T g, dg;
                    gfun(q, cs, g, dg);
                    pc[p] = cs;
                    pg[p] = g;
                    pdg[p] = dg;
                    zj_acc += fc[k] * g;
                    zeta[k] += fc[j] * g;
                }
            }
            zeta[j] += zj_acc;
        }
    }
    // pass 2: bond orders, energy, radial terms, prefactors
    T pref[RMAX], Px[RMAX], Py[RMAX], Pz[RMAX];
#pragma unroll
    for (int j = 0; j < RMAX; ++j) {
        pref[j] = Px[j] = Py[j] = Pz[j] = (T)0;
        if (act[j]) {
            const T z = zeta[j], s = sr[j];
            T bij = (T)1, dbij = (T)0;
            if (z > (T)0) {
                const T x = M<T>::ex(q.n * M<T>::lg(q.beta * z));
                if (x < (T)(1.0 / 1024.0)) {
                    // (1 + x)^(-1/2n) by its series: log1p(x) to x^4 and
                    // exp(-u) to u^3 (truncation below 1e-13 relative)
                    const T l = x * ((T)1 - x * ((T)0.5 - x * ((T)(1.0 / 3.0) - x * (T)0.25)));
                    const T u = q.inv2n * l;
                    bij = (T)1 - u * ((T)1 - u * ((T)0.5 - u * (T)(1.0 / 6.0)));
                } else {
                    bij = M<T>::ex(-q.inv2n * M<T>::l1p(x));
                }
                dbij = (T)(-0.5) * bij * x / (((T)1 + x) * z);
            }
            const T fr = q.AeR * M<T>::ex(-q.l1 * s);
            const T fa = -q.BeR * M<T>::ex(-q.l2 * s);
            const T dfr = -q.l1 * fr, dfa = -q.l2 * fa;
            U += (T)0.5 * fc[j] * (fr + bij * fa);
            const T radial = (T)0.5 * (dfc[j] * (fr + bij * fa) + fc[j] * (dfr + bij * dfa)) * ir[j];
            pref[j] = (T)0.5 * fc[j] * fa * dbij;
            Px[j] = radial * rx[j];
            Py[j] = radial * ry[j];
            Pz[j] = radial * rz[j];
        }
    }
    // pass 3: angular terms, both bonds of each unordered pair at once
    {
        int p = 0;
#pragma unroll
        for (int j = 0; j < RMAX; ++j) {
            T Pxj = 0, Pyj = 0, Pzj = 0;
#pragma unroll
            for (int k = j + 1; k < RMAX; ++k, ++p) {
                if (act[j] && act[k] && (pref[j] != (T)0 || pref[k] != (T)0)) {
                    const T ijk = ir[j] * ir[k];
                    const T cs = pc[p], g = pg[p], dg = pdg[p];
                    const T aj = cs * ir[j] * ir[j], ak = cs * ir[k] * ir[k];
                    const T S = dg * (pref[j] * fc[k] + pref[k] * fc[j]);
                    const T rj = pref[k] * dfc[j] * g * ir[j], rk = pref[j] * dfc[k] * g * ir[k];
                    Pxj += S * (rx[k] * ijk - aj * rx[j]) + rj * rx[j];
                    Pyj += S * (ry[k] * ijk - aj * ry[j]) + rj * ry[j];
                    Pzj += S * (rz[k] * ijk - aj * rz[j]) + rj * rz[j];
                    Px[k] += S * (rx[j] * ijk - ak * rx[k]) + rk * rx[k];
                    Py[k] += S * (ry[j] * ijk - ak * ry[k]) + rk * ry[k];
                    Pz[k] += S * (rz[j] * ijk - ak * rz[k]) + rk * rz[k];
                }
            }
            Px[j] += Pxj;
            Py[j] += Pyj;
            Pz[j] += Pzj;
        }
    }
#pragma unroll
    for (int j = 0; j < RMAX; ++j) {
        if (j < cnt) {
            typename Vec4<T>::type pv;
            pv.x = Px[j];
            pv.y = Py[j];
            pv.z = Pz[j];
            pv.w = (T)0;
            nP[(size_t)j * n + t] = pv;
            // V_mn -= r_m P_n
            vir[0] -= rx[j] * Px[j]; vir[1] -= rx[j] * Py[j]; vir[2] -= rx[j] * Pz[j];
            vir[3] -= ry[j] * Px[j]; vir[4] -= ry[j] * Py[j]; vir[5] -= ry[j] * Pz[j];
            vir[6] -= rz[j] * Px[j]; vir[7] -= rz[j] * Py[j]; vir[8] -= rz[j] * Pz[j];
        }
    }
}

// One thread per atom.  FP32: the records of an atom with at most RMAX list
// entries live in registers (ters_site_reg); more entries take a local
// array.  FP64: the records sit in shared memory, strided by the block size
// so that the threads of a warp hit distinct banks (local memory beyond
// NShared entries).
// MINB: resident blocks per SM the register allocation is held to (FP32;
// picked by the autotuner with the bin width)
template <typename T, int MINB>
__global__ void __launch_bounds__(TILE, MINB) k_ters_partials(const Tile *tiles, BandDev *bands) {
    constexpr bool REG = sizeof(T) == 4;
    constexpr int NS = REG ? 1 : NShared<T>::value;
    Tile tl = tiles[blockIdx.x];
    BandDev &b = bands[tl.band];
    const ImgScalars &sc = b.sc[tl.img];
    __shared__ T s_bv[9], s_dh[9];
    __shared__ int s_nb[3];
    __shared__ TP<T> s_q;  // per-band constants, staged by the whole block
    __shared__ T s_rec[REG ? 1 : NB_FIELDS * NS * TILE];
    if (threadIdx.x < 9) {
        s_bv[threadIdx.x] = (T)sc.bv[threadIdx.x];
        s_dh[threadIdx.x] = (T)sc.dh[threadIdx.x];
    }
    if (threadIdx.x < 3) s_nb[threadIdx.x] = sc.nb[threadIdx.x];
    stage_copy(&s_q, &tp_of<T>(*b.bp));
    __syncthreads();
    const TP<T> &q = s_q;
    const int n = b.n;
    const int t = tl.t * TILE + threadIdx.x;
    const size_t base = (size_t)tl.img * n;
    typename Vec4<T>::type *nP =
        (typename Vec4<T>::type *)b.nbr_P + (size_t)tl.img * MAXN_TERSOFF * n;
    int nin = 0;
    T U = 0;
    T vir[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (t < n) {
        const int cnt = b.nbr_cnt[base + t];
        if (REG && cnt <= RMAX) {
            T rx[RMAX], ry[RMAX], rz[RMAX], sr[RMAX];
            ters_load_reg<T>(q, b, tl.img, t, cnt, s_bv, s_dh, s_nb, rx, ry, rz, sr);
#pragma unroll
            for (int k = 0; k < RMAX; ++k) nin += k < cnt && sub_rn(sr[k], q.D) < q.Dlo;
            ters_site_reg<T>(q, rx, ry, rz, sr, nP, cnt, n, t, U, vir);
        } else if (!REG && cnt <= NS) {
            const Nbr<T> nb{s_rec + threadIdx.x, TILE, NS};
            ters_load<T>(q, b, tl.img, t, cnt, s_bv, s_dh, s_nb, nb);
            for (int k = 0; k < cnt; ++k) nin += sub_rn(nb(NB_SR, k), q.D) < q.Dlo;
            ters_site<T>(q, cnt, nb, nP, n, t, U, vir);
        } else {
            T rec[NB_FIELDS * MAXN_TERSOFF];
            const Nbr<T> nb{rec, 1, MAXN_TERSOFF};
            ters_load<T>(q, b, tl.img, t, cnt, s_bv, s_dh, s_nb, nb);
            for (int k = 0; k < cnt; ++k) nin += sub_rn(nb(NB_SR, k), q.D) < q.Dlo;
            ters_site<T>(q, cnt, nb, nP, n, t, U, vir);
        }
    }
    T acc[12];
    acc[0] = U;
    for (int k = 0; k < 9; ++k) acc[1 + k] = vir[k];
    acc[10] = (T)nin;
    acc[11] = (T)(nin * (nin - 1));
    block_sum_store_tr<12, T>(acc, b.atom_part + ((size_t)tl.img * b.atpi + tl.t) * NPART);
}

// Reverse entries of a rebuilt list: for entry k of slot t (neighbour slot
// qs, stencil code c), the entry of qs's list that points back to t under
// -c, so that the force gather needs no search.
template <typename T>
__device__ inline void ters_reverse_atom(BandDev &b, const Tile &tl, int t) {
    const int n = b.n;
    const size_t base = (size_t)tl.img * n;
    const int *nslot = b.nbr_slot + (size_t)tl.img * MAXN_TERSOFF * n;
    const int *ncode = b.nbr_code + (size_t)tl.img * MAXN_TERSOFF * n;
    unsigned char *nrev = b.nbr_rev + (size_t)tl.img * MAXN_TERSOFF * n;
    const int cnt = b.nbr_cnt[base + t];
    for (int k = 0; k < cnt; ++k) {
        const int qs = nslot[(size_t)k * n + t];
        const int back = neg_code(ncode[(size_t)k * n + t]);
        const int cq = b.nbr_cnt[base + qs];
        int r = 255;
        for (int k2 = 0; k2 < cq; ++k2)
            if (nslot[(size_t)k2 * n + qs] == t && ncode[(size_t)k2 * n + qs] == back) {
                r = k2;
                break;
            }
        nrev[(size_t)k * n + t] = (unsigned char)r;
    }
}

template <typename T>
__global__ void __launch_bounds__(TILE) k_ters_reverse(const Tile *tiles, int ntiles, BandDev *bands) {
    for (int k = blockIdx.x; k < ntiles; k += gridDim.x) {
        const Tile tl = tiles[k];
        BandDev &b = bands[tl.band];
        if (!b.sc[tl.img].rebuild) continue;
        const int t = tl.t * TILE + threadIdx.x;
        if (t < b.n) ters_reverse_atom<T>(b, tl, t);
    }
}

template <typename T>
__global__ void __launch_bounds__(TILE) k_ters_gather(const Tile *tiles, BandDev *bands) {
    using T4 = typename Vec4<T>::type;
    const Tile tl = tiles[blockIdx.x];
    const BandDev &b = bands[tl.band];
    const int n = b.n;
    const int t = tl.t * TILE + threadIdx.x;
    if (t >= n) return;
    const size_t base = (size_t)tl.img * n;
    const int *nslot = b.nbr_slot + (size_t)tl.img * MAXN_TERSOFF * n;
    const unsigned char *nrev = b.nbr_rev + (size_t)tl.img * MAXN_TERSOFF * n;
    const T4 *nP = (const T4 *)b.nbr_P + (size_t)tl.img * MAXN_TERSOFF * n;
    const int cnt = b.nbr_cnt[base + t];
    const int atom = b.slot_atom[base + t];
    // f^ij = P_ij - P_ji, in list order.  The first GK entries: their
    // indices, then every partial they point to, are loaded before any is
    // used (two round trips for the atom, not one per entry).
    constexpr int GK = 4;
    int qs[GK], k2[GK];
#pragma unroll
    for (int k = 0; k < GK; ++k) {
        qs[k] = k < cnt ? nslot[(size_t)k * n + t] : 0;
        k2[k] = k < cnt ? nrev[(size_t)k * n + t] : 255;
    }
    T ax[GK], ay[GK], az[GK], rx[GK], ry[GK], rz[GK];
#pragma unroll
    for (int k = 0; k < GK; ++k) {
        ax[k] = ay[k] = az[k] = rx[k] = ry[k] = rz[k] = (T)0;
        if (k < cnt) {
            const T4 a = nP[(size_t)k * n + t];
            ax[k] = a.x;
            ay[k] = a.y;
            az[k] = a.z;
        }
        if (k2[k] != 255) {
            const T4 r = nP[(size_t)k2[k] * n + qs[k]];
            rx[k] = r.x;
            ry[k] = r.y;
            rz[k] = r.z;
        }
    }
    T fx = 0, fy = 0, fz = 0;
#pragma unroll
    for (int k = 0; k < GK; ++k) {
        if (k < cnt) {
            fx += ax[k];
            fy += ay[k];
            fz += az[k];
            if (k2[k] != 255) {
                fx -= rx[k];
                fy -= ry[k];
                fz -= rz[k];
            }
        }
    }
    for (int k = GK; k < cnt; ++k) {
        const T4 a = nP[(size_t)k * n + t];
        fx += a.x;
        fy += a.y;
        fz += a.z;
        const int q = nslot[(size_t)k * n + t];
        const int r = nrev[(size_t)k * n + t];
        if (r != 255) {
            const T4 p = nP[(size_t)r * n + q];
            fx -= p.x;
            fy -= p.y;
            fz -= p.z;
        }
    }
    // D in T: the FP32 leading part k_mapback / the move stored (FP32
    // bands), or D itself (FP64 bands); no conversion in this kernel
    const ImgScalars &sc = b.sc[tl.img];
    T D[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) D[k] = sizeof(T) == 4 ? (T)sc.dfl[k] : (T)sc.D[k];
    const T g0 = fx * D[0] + fy * D[1] + fz * D[2];
    const T g1 = fx * D[3] + fy * D[4] + fz * D[5];
    const T g2 = fx * D[6] + fy * D[7] + fz * D[8];
    T *F = (T *)b.F + ((size_t)tl.img * b.rows + atom) * 3;
    F[0] = g0;
    F[1] = g1;
    F[2] = g2;
}

// ---- NEP-style potential: descriptors and a neural-network site energy ----
//
// U_i = sum_h w1_h tanh(sum_d W0_hd q_d - b0_h) - b1 over the descriptors of
// i's neighbours within rc (single species): radial q_n = sum_j g^R_n(r_ij)
// and angular q_nl = sum_jk g^A_n(r_ij) g^A_n(r_ik) P_l(cos theta_jk), l =
// 1..4, with g^{R,A}_n = sum_k c_nk f_k, f_k = (T_k(x) + 1)/2 f_c(r),
// x = 2 (r/rc - 1)^2 - 1 (Chebyshev T_k) and f_c = cos^2(pi r / 2rc) (=
// (1 + cos(pi r/rc))/2, written without cancellation near rc).  The paper's
// examples use a neuroevolution potential of this form (Sec. IV); trained
// weights are not available, so the caller passes synthetic ones.
//
// The kernel reuses the many-body machinery of the Tersoff path: the same
// neighbour lists (entries within rc + skin), the same compensated pair
// vectors (s = r - rc), per-entry partials P_ij = dU_i/dr^ij written for the
// deterministic reverse-entry gather, and the site virial.  The angular
// sums run over unordered neighbour pairs (cos, P_l and P_l' symmetric).

enum { NE_IR = NB_SR + 1, NE_GA, NE_DGA = NE_GA + NEP_NA, NE_PX = NE_DGA + NEP_NA, NE_PY, NE_PZ,
       NE_FIELDS };

__device__ inline void sincospi_t(float x, float *s, float *c) { sincospif(x, s, c); }
__device__ inline void sincospi_t(double x, double *s, double *c) { sincospi(x, s, c); }
__device__ inline float tanh_t(float x) { return tanhf(x); }
__device__ inline double tanh_t(double x) { return tanh(x); }

template <typename T> __device__ inline const T *nep_weights(const BandDev &b);
template <> __device__ inline const float *nep_weights<float>(const BandDev &b) { return b.nep_wf; }
template <> __device__ inline const double *nep_weights<double>(const BandDev &b) { return b.nep_w; }

// f_k(r) and f_k'(r), k < NEP_K
template <typename T>
__device__ inline void nep_basis(T r, T inv_rc, T *f, T *df) {
    T sh, ch;
    sincospi_t((T)0.5 * r * inv_rc, &sh, &ch);
    const T fc = ch * ch, dfc = -(T)3.14159265358979323846 * inv_rc * sh * ch;
    const T u = r * inv_rc - (T)1;
    const T x = (T)2 * u * u - (T)1, dx = (T)4 * u * inv_rc;
    T t0 = (T)1, t1 = x, d0 = (T)0, d1 = (T)1;  // T_k(x), dT_k/dx
    f[0] = fc;
    df[0] = dfc;
    f[1] = (T)0.5 * (x + (T)1) * fc;
    df[1] = (T)0.5 * (dx * fc + (x + (T)1) * dfc);
#pragma unroll
    for (int k = 2; k < NEP_K; ++k) {
        const T t2 = (T)2 * x * t1 - t0, d2 = (T)2 * t1 + (T)2 * x * d1 - d0;
        f[k] = (T)0.5 * (t2 + (T)1) * fc;
        df[k] = (T)0.5 * (d2 * dx * fc + (t2 + (T)1) * dfc);
        t0 = t1; t1 = t2; d0 = d1; d1 = d2;
    }
}

// P_1..P_4 and their derivatives
template <typename T>
__device__ inline void nep_legendre(T c, T *P, T *dP) {
    const T c2 = c * c;
    P[0] = c;                                   dP[0] = (T)1;
    P[1] = (T)1.5 * c2 - (T)0.5;                dP[1] = (T)3 * c;
    P[2] = ((T)2.5 * c2 - (T)1.5) * c;          dP[2] = (T)7.5 * c2 - (T)1.5;
    P[3] = ((T)4.375 * c2 - (T)3.75) * c2 + (T)0.375;
    dP[3] = ((T)17.5 * c2 - (T)7.5) * c;
}

template <typename T>
__device__ inline void nep_site(const TP<T> &q, const T *w, int cnt, const Nbr<T> &nb,
                                typename Vec4<T>::type *nP, int n, int t, T &U, T (&vir)[9],
                                int &nin) {
    const T rc = q.R, inv_rc = (T)1 / q.R;
    T qd[NEP_ND];
#pragma unroll
    for (int d = 0; d < NEP_ND; ++d) qd[d] = (T)0;
    // pass 0: radial descriptors, angular radial functions
    for (int j = 0; j < cnt; ++j) {
        const T s = nb(NB_SR, j);
        if (!(s < (T)0)) {  // at or beyond rc: no terms
            nb(NE_IR, j) = (T)0;
            continue;
        }
        ++nin;
        const T r = rc + s;
        T f[NEP_K], df[NEP_K];
        nep_basis(r, inv_rc, f, df);
#pragma unroll
        for (int m = 0; m < NEP_NR; ++m) {
            T g = 0;
#pragma unroll
            for (int k = 0; k < NEP_K; ++k) g += w[NEP_OCR + m * NEP_K + k] * f[k];
            qd[m] += g;
        }
#pragma unroll
        for (int m = 0; m < NEP_NA; ++m) {
            T g = 0, dg = 0;
#pragma unroll
            for (int k = 0; k < NEP_K; ++k) {
                g += w[NEP_OCA + m * NEP_K + k] * f[k];
                dg += w[NEP_OCA + m * NEP_K + k] * df[k];
            }
            nb(NE_GA + m, j) = g;
            nb(NE_DGA + m, j) = dg;
        }
        nb(NE_IR, j) = M<T>::rcp(r);
    }
    // pass 1: angular descriptors (j = k terms: P_l(1) = 1)
    for (int j = 0; j < cnt; ++j) {
        const T irj = nb(NE_IR, j);
        if (irj == (T)0) continue;
        const T xj = nb(NB_RX, j), yj = nb(NB_RY, j), zj = nb(NB_RZ, j);
        T gj[NEP_NA];
#pragma unroll
        for (int m = 0; m < NEP_NA; ++m) {
            gj[m] = nb(NE_GA + m, j);
#pragma unroll
            for (int l = 0; l < NEP_L; ++l) qd[NEP_NR + m * NEP_L + l] += gj[m] * gj[m];
        }
        for (int k = j + 1; k < cnt; ++k) {
            const T irk = nb(NE_IR, k);
            if (irk == (T)0) continue;
            const T c = (xj * nb(NB_RX, k) + yj * nb(NB_RY, k) + zj * nb(NB_RZ, k)) * irj * irk;
            T P[NEP_L], dP[NEP_L];
            nep_legendre(c, P, dP);
#pragma unroll
            for (int m = 0; m < NEP_NA; ++m) {
                const T pr = (T)2 * gj[m] * nb(NE_GA + m, k);
#pragma unroll
                for (int l = 0; l < NEP_L; ++l) qd[NEP_NR + m * NEP_L + l] += pr * P[l];
            }
        }
    }
    // the network and dU/dq
    T dU[NEP_ND];
#pragma unroll
    for (int d = 0; d < NEP_ND; ++d) dU[d] = (T)0;
    T Ui = -w[NEP_OB1];
    for (int h = 0; h < NEP_H; ++h) {
        T a = -w[NEP_OB0 + h];
#pragma unroll
        for (int d = 0; d < NEP_ND; ++d) a += w[NEP_OW0 + h * NEP_ND + d] * qd[d];
        const T th = tanh_t(a);
        Ui += w[NEP_OW1 + h] * th;
        const T co = w[NEP_OW1 + h] * ((T)1 - th * th);
#pragma unroll
        for (int d = 0; d < NEP_ND; ++d) dU[d] += co * w[NEP_OW0 + h * NEP_ND + d];
    }
    U += Ui;
    // sum_l dU/dq_ml, for the j = k terms
    T dUs[NEP_NA];
#pragma unroll
    for (int m = 0; m < NEP_NA; ++m) {
        dUs[m] = 0;
#pragma unroll
        for (int l = 0; l < NEP_L; ++l) dUs[m] += dU[NEP_NR + m * NEP_L + l];
    }
    // pass 3a: coefficient of r^_j from the radial terms and the j = k terms
    // (kept in the s field, no longer needed), partials zeroed
    for (int j = 0; j < cnt; ++j) {
        nb(NE_PX, j) = nb(NE_PY, j) = nb(NE_PZ, j) = (T)0;
        const T irj = nb(NE_IR, j);
        if (irj == (T)0) {
            nb(NB_SR, j) = (T)0;
            continue;
        }
        T f[NEP_K], df[NEP_K];
        nep_basis(rc + nb(NB_SR, j), inv_rc, f, df);
        T alpha = 0;
#pragma unroll
        for (int m = 0; m < NEP_NR; ++m) {
            T dg = 0;
#pragma unroll
            for (int k = 0; k < NEP_K; ++k) dg += w[NEP_OCR + m * NEP_K + k] * df[k];
            alpha += dU[m] * dg;
        }
#pragma unroll
        for (int m = 0; m < NEP_NA; ++m)
            alpha += (T)2 * nb(NE_GA + m, j) * nb(NE_DGA + m, j) * dUs[m];
        nb(NB_SR, j) = alpha;
    }
    // pass 3b: pairs j < k
    for (int j = 0; j < cnt; ++j) {
        const T irj = nb(NE_IR, j);
        if (irj == (T)0) continue;
        const T xj = nb(NB_RX, j) * irj, yj = nb(NB_RY, j) * irj, zj = nb(NB_RZ, j) * irj;
        T gj[NEP_NA], dgj[NEP_NA];
#pragma unroll
        for (int m = 0; m < NEP_NA; ++m) {
            gj[m] = nb(NE_GA + m, j);
            dgj[m] = nb(NE_DGA + m, j);
        }
        T aj = 0, Pxj = 0, Pyj = 0, Pzj = 0;
        for (int k = j + 1; k < cnt; ++k) {
            const T irk = nb(NE_IR, k);
            if (irk == (T)0) continue;
            const T xk = nb(NB_RX, k) * irk, yk = nb(NB_RY, k) * irk, zk = nb(NB_RZ, k) * irk;
            const T c = xj * xk + yj * yk + zj * zk;
            T P[NEP_L], dP[NEP_L];
            nep_legendre(c, P, dP);
            T ak = 0, B = 0;
#pragma unroll
            for (int m = 0; m < NEP_NA; ++m) {
                T S = 0, Tm = 0;
#pragma unroll
                for (int l = 0; l < NEP_L; ++l) {
                    S += dU[NEP_NR + m * NEP_L + l] * P[l];
                    Tm += dU[NEP_NR + m * NEP_L + l] * dP[l];
                }
                const T gk = nb(NE_GA + m, k), dgk = nb(NE_DGA + m, k);
                aj += (T)2 * dgj[m] * gk * S;
                ak += (T)2 * dgk * gj[m] * S;
                B += (T)2 * gj[m] * gk * Tm;
            }
            // d cos / d r^ij = (r^_ik - cos r^_ij) / r_ij (and j <-> k)
            const T bj = B * irj, bk = B * irk;
            Pxj += bj * (xk - c * xj);
            Pyj += bj * (yk - c * yj);
            Pzj += bj * (zk - c * zj);
            nb(NB_SR, k) += ak;
            nb(NE_PX, k) += bk * (xj - c * xk);
            nb(NE_PY, k) += bk * (yj - c * yk);
            nb(NE_PZ, k) += bk * (zj - c * zk);
        }
        nb(NB_SR, j) += aj;
        nb(NE_PX, j) += Pxj;
        nb(NE_PY, j) += Pyj;
        nb(NE_PZ, j) += Pzj;
    }
    // pass 4: P_ij = (alpha_j r^_ij + angular terms), partials out, virial
    for (int j = 0; j < cnt; ++j) {
        const T irj = nb(NE_IR, j), alpha = nb(NB_SR, j);
        const T rx = nb(NB_RX, j), ry = nb(NB_RY, j), rz = nb(NB_RZ, j);
        const T Px = nb(NE_PX, j) + alpha * rx * irj, Py = nb(NE_PY, j) + alpha * ry * irj,
                Pz = nb(NE_PZ, j) + alpha * rz * irj;
        typename Vec4<T>::type pv;
        pv.x = Px;
        pv.y = Py;
        pv.z = Pz;
        pv.w = (T)0;
        nP[(size_t)j * n + t] = pv;
        vir[0] -= rx * Px; vir[1] -= rx * Py; vir[2] -= rx * Pz;
        vir[3] -= ry * Px; vir[4] -= ry * Py; vir[5] -= ry * Pz;
        vir[6] -= rz * Px; vir[7] -= rz * Py; vir[8] -= rz * Pz;
    }
}

// One thread per atom, records in shared memory (local memory past NS
// entries), weights staged per block.
template <typename T>
__global__ void __launch_bounds__(TILE, sizeof(T) == 4 ? 4 : 1) k_nep_partials(const Tile *tiles, BandDev *bands) {
    // records of up to 6 (FP32) or 3 (FP64) entries per atom in shared
    // memory: 12 fields each, within the 48 KB of static shared memory
    constexpr int NS = sizeof(T) == 4 ? 6 : 3;
    Tile tl = tiles[blockIdx.x];
    BandDev &b = bands[tl.band];
    const ImgScalars &sc = b.sc[tl.img];
    __shared__ T s_bv[9], s_dh[9];
    __shared__ int s_nb[3];
    __shared__ TP<T> s_q;
    __shared__ T s_w[NEP_NW];
    __shared__ T s_rec[NE_FIELDS * NS * TILE];
    if (threadIdx.x < 9) {
        s_bv[threadIdx.x] = (T)sc.bv[threadIdx.x];
        s_dh[threadIdx.x] = (T)sc.dh[threadIdx.x];
    }
    if (threadIdx.x < 3) s_nb[threadIdx.x] = sc.nb[threadIdx.x];
    stage_copy(&s_q, &tp_of<T>(*b.bp));
    const T *wg = nep_weights<T>(b);
    for (int k = threadIdx.x; k < NEP_NW; k += TILE) s_w[k] = wg[k];
    __syncthreads();
    const TP<T> &q = s_q;
    const int n = b.n;
    const int t = tl.t * TILE + threadIdx.x;
    const size_t base = (size_t)tl.img * n;
    typename Vec4<T>::type *nP =
        (typename Vec4<T>::type *)b.nbr_P + (size_t)tl.img * MAXN_TERSOFF * n;
    int nin = 0;
    T U = 0;
    T vir[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (t < n) {
        const int cnt = b.nbr_cnt[base + t];
        if (cnt <= NS) {
            const Nbr<T> nb{s_rec + threadIdx.x, TILE, NS};
            ters_load<T>(q, b, tl.img, t, cnt, s_bv, s_dh, s_nb, nb);
            nep_site<T>(q, s_w, cnt, nb, nP, n, t, U, vir, nin);
        } else {
            T rec[NE_FIELDS * MAXN_TERSOFF];
            const Nbr<T> nb{rec, 1, MAXN_TERSOFF};
            ters_load<T>(q, b, tl.img, t, cnt, s_bv, s_dh, s_nb, nb);
            nep_site<T>(q, s_w, cnt, nb, nP, n, t, U, vir, nin);
        }
    }
    T acc[12];
    acc[0] = U;
    for (int k = 0; k < 9; ++k) acc[1 + k] = vir[k];
    acc[10] = (T)nin;
    acc[11] = (T)(nin * (nin - 1));
    block_sum_store<12, T>(acc, b.atom_part + ((size_t)tl.img * b.atpi + tl.t) * NPART);
}

template <typename T>
void launch_tersoff_list(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s) {
    if (ntiles <= 0) return;
    k_ters_list<T><<<ntiles < gated_grid() ? ntiles : gated_grid(), TILE, 0, s>>>(tiles, ntiles, bands);
}
template <typename T>
void launch_tersoff_reverse(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s) {
    if (ntiles <= 0) return;
    k_ters_reverse<T><<<ntiles < gated_grid() ? ntiles : gated_grid(), TILE, 0, s>>>(tiles, ntiles,
                                                                                 bands);
}
template <typename T>
void launch_tersoff_partials(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s,
                             int minb) {
    if (ntiles <= 0) return;
    if (sizeof(T) == 8) {
        k_ters_partials<T, 1><<<ntiles, TILE, 0, s>>>(tiles, bands);
        return;
    }
    switch (minb) {
        case 4: k_ters_partials<T, 4><<<ntiles, TILE, 0, s>>>(tiles, bands); break;
        case 6: k_ters_partials<T, 6><<<ntiles, TILE, 0, s>>>(tiles, bands); break;
        case 7: k_ters_partials<T, 7><<<ntiles, TILE, 0, s>>>(tiles, bands); break;
        case 8: k_ters_partials<T, 8><<<ntiles, TILE, 0, s>>>(tiles, bands); break;
        default: k_ters_partials<T, 5><<<ntiles, TILE, 0, s>>>(tiles, bands); break;
    }
}
template <typename T>
void launch_tersoff_gather(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s) {
    if (ntiles <= 0) return;
    k_ters_gather<T><<<ntiles, TILE, 0, s>>>(tiles, bands);
}
template void launch_tersoff_list<float>(const Tile *, int, BandDev *, cudaStream_t);
template void launch_tersoff_list<double>(const Tile *, int, BandDev *, cudaStream_t);
template void launch_tersoff_reverse<float>(const Tile *, int, BandDev *, cudaStream_t);
template void launch_tersoff_reverse<double>(const Tile *, int, BandDev *, cudaStream_t);
template void launch_tersoff_partials<float>(const Tile *, int, BandDev *, cudaStream_t, int);
template void launch_tersoff_partials<double>(const Tile *, int, BandDev *, cudaStream_t, int);
template <typename T>
void launch_nep_partials(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s) {
    if (ntiles <= 0) return;
    k_nep_partials<T><<<ntiles, TILE, 0, s>>>(tiles, bands);
}
template void launch_nep_partials<float>(const Tile *, int, BandDev *, cudaStream_t);
template void launch_nep_partials<double>(const Tile *, int, BandDev *, cudaStream_t);
template void launch_tersoff_gather<float>(const Tile *, int, BandDev *, cudaStream_t);
template void launch_tersoff_gather<double>(const Tile *, int, BandDev *, cudaStream_t);

}  // namespace cfneb
