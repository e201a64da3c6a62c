// Per-image reduction, cell-filter lattice force, NEB projection and FIRE.
//
// k_image_finalize  sums the force kernel's tile partials (FP64, slot order)
//                   into E and V, adds the external pressure (H = U + P Omega,
//                   V - P Omega I) and writes the three lattice rows of the
//                   generalised force: (1/c) 1/2 D^-T V_sym D^-1 for the
//                   rotation-free filter, (1/c) D^-T V for the deformation
//                   gradient (Sec. II.C).
// The band phase of a step is three passes over the row tiles of the
// interior images:
// k_band_dots       pass 1: per tile, ten dots with compensated
//                   accumulation (|dX+|^2, |dX-|^2, dX+.dX-, F.dX+, F.dX-,
//                   F.F, F.v, v.v, dX+.v, dX-.v; dX+ = X_{i+1} - X_i,
//                   dX- = X_i - X_{i-1}); the last tile of an image sums the
//                   image's tiles in FP64 and computes the image's upwind
//                   tangent weights, the two coefficients of
//                   f_NEB = F + a dX+ + b dX- (Sec. II.A; the climbing image
//                   is the argmax of the energies, final before this pass)
//                   and its FIRE terms F_NEB.v, |F_NEB|^2, |v|^2 from the dots.
// k_neb_force       pass 2: writes f_NEB and takes the largest row norm; the
//                   last tile of a band sums the images' FIRE terms, runs the
//                   convergence test and the FIRE decision (Bitzek et al.
//                   2006, band-global power).
// k_fire_update     pass 3: v <- cv v + cf F; v += dt F; dX = dt v clamped
//                   per row to maxstep; X += dX (interior images only); with
//                   a skin, also each row tile's largest displacement since
//                   the last list build (the next step's reuse test).  One
//                   warp per image moves its lattice rows and computes the
//                   new cell for the next map-back, beside the row tiles.
// "Last" blocks are found with completion counters (an acquire-release
// atomic increment); the sums they form read the other blocks' records in a
// fixed order, so results do not depend on block scheduling.
#include "common.cuh"

namespace cfneb {

template <typename T>
__global__ void __launch_bounds__(FIN_THREADS) k_image_finalize(const ImgRef *imgs, BandDev *bands) {
    ImgRef r = imgs[blockIdx.x];
    BandDev &b = bands[r.band];
    const BandParams *bp = b.bp;
    ImgScalars &sc = b.sc[r.img];
    // U, V (9), pairs, triples: tile partials summed in FP64, fixed order
    __shared__ double s_tot[12];
    const double tk = block_sum_records_wide<12, 12, FIN_THREADS, false>(
        b.atom_part + (size_t)r.img * b.atpi * NPART, NPART, b.atpi);
    if (threadIdx.x < 12) s_tot[threadIdx.x] = tk;
    __syncthreads();
    if (threadIdx.x >= 32) return;
    // warp 0: the 3x3 work lane-parallel (lane l holds entry (l / 3, l % 3))
    const Lane3 p;
    const int lane = threadIdx.x;
    const double P = bp->pressure, omega = sc.omega;
    double V = s_tot[1 + p.l];
    if (P != 0.0 && p.i == p.j) V -= P * omega;
    if (lane == 0) {
        sc.pairs = s_tot[10];
        sc.triples = s_tot[11];
        sc.U = s_tot[0];
        sc.E = P != 0.0 ? s_tot[0] + P * omega : s_tot[0];
    }
    if (lane < 9) sc.V[lane] = V;
    double Phi = 0.0;
    if (bp->filter) {
        const double Di = sc.Dinv[p.l];
        const double DiT = ltrans(Di, p);
        if (bp->variant == 0) {
            const double Vs = 0.5 * (V + ltrans(V, p));
            Phi = lmul(lmul(DiT, Vs, p), Di, p) * (0.5 * rcp64(bp->c));
        } else {
            Phi = lmul(DiT, V, p) * rcp64(bp->c);
        }
    }
    T *F = (T *)b.F + ((size_t)r.img * b.rows + b.n) * 3;
    if (lane < 9) F[lane] = (T)Phi;
}

// ---- band pass 1: the ten dot products of every interior image ------------
//
// Row sums in T, accumulated across rows with Knuth's two-sum (FP32: the
// running sum is carried as an unevaluated pair s + c, so the error of a
// thread's total is the rounding of each row's 3-term product sum,
// |err| <= 2^-23 sum_rows sum_c |a_c b_c|, with no growth in the row count);
// the warp butterfly adds pairs the same way and the block total is formed
// in FP64 from the pairs.  FP64 bands accumulate plainly in FP64.
template <typename T> struct Acc;
template <> struct Acc<float> {
    float s = 0.0f, c = 0.0f;
    __device__ void add(float p) {
        const float t = __fadd_rn(s, p), z = __fsub_rn(t, s);
        c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z)));
        s = t;
    }
    __device__ void add(const Acc &o) {  // pair + pair
        add(o.s);
        c = __fadd_rn(c, o.c);
    }
    __device__ Acc shfl(int o) const {  // the partner lane's pair
        Acc q;
        q.s = __shfl_xor_sync(0xffffffffu, s, o);
        q.c = __shfl_xor_sync(0xffffffffu, c, o);
        return q;
    }
    __device__ double value() const { return (double)s + (double)c; }
};
template <> struct Acc<double> {
    double s = 0.0;
    __device__ void add(double p) { s += p; }
    __device__ void add(const Acc &o) { s += o.s; }
    __device__ Acc shfl(int o) const {
        Acc q;
        q.s = __shfl_xor_sync(0xffffffffu, s, o);
        return q;
    }
    __device__ double value() const { return s; }
};

// Block totals of K accumulators in a fixed order: a transposing butterfly
// within each warp (at each level a lane keeps half of its values and adds
// its partner's copy of them, so 16 values take 31 exchanges instead of 80,
// and lane 2j ends with value j), then warps 0..7 in turn.  Thread 0 stores
// the totals to dst[0..K-1] in FP64.
template <int K, typename T>
__device__ inline void block_acc_store(Acc<T> (&v)[K], double *dst) {
    static_assert(K <= 16, "values are padded to 16");
    __shared__ Acc<T> red[RTHREADS / 32][16];
    __shared__ double s_tot[16];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    Acc<T> a[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = k < K ? v[k] : Acc<T>();
#pragma unroll
    for (int h = 8, o = 16; h >= 1; h >>= 1, o >>= 1) {
        const bool hi = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < h; ++k) {
            const Acc<T> send = hi ? a[k] : a[k + h];
            Acc<T> keep = hi ? a[k + h] : a[k];
            keep.add(send.shfl(o));
            a[k] = keep;
        }
    }
    a[0].add(a[0].shfl(1));
    if ((lane & 1) == 0) red[w][lane >> 1] = a[0];
    __syncthreads();
    if (threadIdx.x < K) {
        Acc<T> t = red[0][threadIdx.x];
        for (int q = 1; q < RTHREADS / 32; ++q) t.add(red[q][threadIdx.x]);
        s_tot[threadIdx.x] = t.value();
    }
    __syncthreads();
    // thread 0 stores the record: its increment of the image's counter
    // (last_arrival) publishes it to the block that finishes the image
    if (threadIdx.x == 0)
        for (int k = 0; k < K; ++k) dst[k] = s_tot[k];
    __syncthreads();
}

// true in every thread of the one block that arrives last (counter reaches
// total); that block also resets the counter for the next launch.  Writes
// the other blocks must see are thread 0's, made before the call
// (thread 0's increment is an acquire-release atomic at GPU scope: its
// release publishes the record thread 0 stored before it, its acquire in
// the last block orders the reads of the other blocks' records after it,
// and the barrier passes that order to the block's other threads)
__device__ inline unsigned atom_add_acq_rel(unsigned int *p, unsigned int v) {
    unsigned int old;
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ inline bool last_arrival(unsigned int *counter, unsigned int total) {
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int prev = atom_add_acq_rel(counter, 1u);
        s_last = prev + 1u == total;
        if (s_last) *counter = 0u;
    }
    __syncthreads();
    return s_last != 0;
}

// Climbing image of a band: argmax of the step energies over the interior
// images, lowest index on ties (the energies are final before pass 1).
// Called by a whole warp with e0 = the energy of image 1 + lane (loaded by
// the caller ahead of other work; -inf where there is no such image): a
// butterfly keeps (larger energy, else lower index), so every lane returns
// the same index.
__device__ inline int climbing_image_warp(const BandDev &b, int N, double e0) {
    const int lane = threadIdx.x & 31;
    double best = -INFINITY;
    int bi = 0x7fffffff;
    if (1 + lane < N - 1 && e0 > best) {  // NaN never wins
        best = e0;
        bi = 1 + lane;
    }
    for (int i = 33 + lane; i < N - 1; i += 32) {
        const double e = __ldcg(&b.sc[i].E);
        if (e > best) {  // i grows within a lane: ties keep the lower index
            best = e;
            bi = i;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double e2 = __shfl_xor_sync(0xffffffffu, best, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
        if (e2 > best || (e2 == best && i2 < bi)) {
            best = e2;
            bi = i2;
        }
    }
    return bi == 0x7fffffff ? 1 : bi;  // all energies NaN: the first image
}

// One image, after its dots: upwind tangent weights and the two
// coefficients with f_NEB = F + a dX+ + b dX-.  Since tau = w+ dX+ + w- dX-,
// |tau| and F.tau follow from five dots, and the projection
// f - (f.t)t + k(|dX+| - |dX-|) t (Sec. II.A; climbing image f - 2 (f.t) t)
// is two scalars per image.  The image's FIRE terms follow from the other
// five dots without a pass over f_NEB:
//   F_NEB.v = F.v + a dX+.v + b dX-.v,
//   |F_NEB|^2 = F.F + a^2 |dX+|^2 + b^2 |dX-|^2 + 2a F.dX+ + 2b F.dX-
//               + 2ab dX+.dX-.
// etol: energy differences up to etol count as ties (0 in FP64 bands: the
// rule exactly as stated; mixed bands: the error bound of their step
// energies, FP32 site energies summed in FP64, so that the upwind branch is
// not chosen by rounding between nearly equal images -- those take the
// equal-weight tangent dX+ + dX-).
__device__ inline void image_coef(BandDev &b, int i, int ci, const double *d, double Em,
                                  double E0, double Ep, double kspring, double etol) {
    ImgScalars &sc = b.sc[i];
    double wp, wm;
    if (Ep - E0 > etol && E0 - Em > etol) {
        wp = 1.0; wm = 0.0;
    } else if (E0 - Ep > etol && Em - E0 > etol) {
        wp = 0.0; wm = 1.0;
    } else {
        const double a = fabs(Ep - E0), c = fabs(Em - E0);
        const double dmax = fmax(a, c), dmin = fmin(a, c);
        if (dmax <= etol) {
            wp = 1.0; wm = 1.0;
        } else if (Ep > Em) {
            wp = dmax; wm = dmin;
        } else {
            wp = dmin; wm = dmax;
        }
    }
    const double pp = d[0], mm = d[1], pm = d[2], fp = d[3], fm = d[4];
    const double tt = wp * wp * pp + 2.0 * wp * wm * pm + wm * wm * mm;
    // 1 / |tau| and the spring lengths from FP32-seeded Newton steps (an FP64
    // divide or square root is a long dependent sequence on this GPU)
    const double itn = rsqrt64(tt);
    const double ft = (wp * fp + wm * fm) * itn;  // F . tau_hat
    const double gamma = i == ci ? -2.0 * ft : kspring * (sqrt64(pp) - sqrt64(mm)) - ft;
    const double a = gamma * wp * itn, bb = gamma * wm * itn;
    sc.coef[0] = a;
    sc.coef[1] = bb;
    sc.fire[0] = d[6] + a * d[8] + bb * d[9];
    sc.fire[1] = d[5] + a * a * pp + bb * bb * mm + 2.0 * a * fp + 2.0 * bb * fm +
                 2.0 * a * bb * pm;
    sc.fire[2] = d[7];
}

// Pass 1 over the row tiles of the interior images: the ten dots of each
// tile into the tile's partial record; with FUSE, the last tile of an image
// sums the image's records (fixed order) into its dots, and the last image
// of a band computes the band's NEB coefficients and FIRE sums.
// Each thread of a row tile owns 4 consecutive rows: 12 values, loaded and
// stored with 16-byte vector accesses (the row stride of an image is a
// multiple of 4 rows, so every thread's first value is 16-byte aligned).
__device__ inline void ld12(const float *p, float (&v)[12]) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float4 a = q[k];
        v[4 * k] = a.x; v[4 * k + 1] = a.y; v[4 * k + 2] = a.z; v[4 * k + 3] = a.w;
    }
}
__device__ inline void ld12(const double *p, double (&v)[12]) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const double2 a = q[k];
        v[2 * k] = a.x; v[2 * k + 1] = a.y;
    }
}
__device__ inline void st12(float *p, const float (&v)[12]) {
    float4 *q = reinterpret_cast<float4 *>(p);
#pragma unroll
    for (int k = 0; k < 3; ++k) q[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
}
__device__ inline void st12(double *p, const double (&v)[12]) {
    double2 *q = reinterpret_cast<double2 *>(p);
#pragma unroll
    for (int k = 0; k < 6; ++k) q[k] = make_double2(v[2 * k], v[2 * k + 1]);
}

template <typename T, bool FUSE>
__global__ void __launch_bounds__(RTHREADS, sizeof(T) == 4 ? 4 : 2) k_band_dots(const Tile *tiles, BandDev *bands) {
    Tile tl = tiles[blockIdx.x];
    BandDev &b = bands[tl.band];
    Acc<T> acc[10];
    const size_t stride = (size_t)b.rows * 3;
    const int r0 = tl.t * RTILE + RPT * (int)threadIdx.x;  // first of this thread's rows
    if (r0 < b.rows) {
        const size_t o0 = tl.img * stride + (size_t)r0 * 3;
        T a[12], xp[12], xm[12], f[12], v[12];
        ld12((const T *)b.X + o0, a);
        ld12((const T *)b.X + o0 + stride, xp);
        ld12((const T *)b.X + o0 - stride, xm);
        ld12((const T *)b.F + o0, f);
        ld12((const T *)b.v + o0, v);
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            T r[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
            for (int c = 3 * q; c < 3 * q + 3; ++c) {
                const T dp = xp[c] - a[c], dm = a[c] - xm[c];
                const T fc = f[c], vc = v[c];
                r[0] = fma(dp, dp, r[0]);
                r[1] = fma(dm, dm, r[1]);
                r[2] = fma(dp, dm, r[2]);
                r[3] = fma(fc, dp, r[3]);
                r[4] = fma(fc, dm, r[4]);
                r[5] = fma(fc, fc, r[5]);
                r[6] = fma(fc, vc, r[6]);
                r[7] = fma(vc, vc, r[7]);
                r[8] = fma(dp, vc, r[8]);
                r[9] = fma(dm, vc, r[9]);
            }
#pragma unroll
            for (int k = 0; k < 10; ++k) acc[k].add(r[k]);
        }
    }
    double *part = b.row_part + ((size_t)tl.img * b.rtpi + tl.t) * NPART;
    block_acc_store<10, T>(acc, part);
    if (!FUSE) return;
    ImgScalars &sc = b.sc[tl.img];
    if (!last_arrival(&sc.done, (unsigned)b.rtpi)) return;
    // warp 0 loads what the climbing image and the tangent need before the
    // record sums, so that those loads share the sums' round trip
    BandParams *bp = b.bp;
    const int lane = threadIdx.x & 31;
    double e0 = 0.0, Em = 0.0, E0 = 0.0, Ep = 0.0, kspring = 0.0;
    int N = 0, climb = 0, shard = 0, ci_ext = -1;
    if (threadIdx.x < 32) {
        if (1 + lane < b.ncap) e0 = __ldcg(&b.sc[1 + lane].E);
        N = bp->N;
        climb = bp->climb;
        shard = bp->shard;
        ci_ext = bp->ci_ext;
        kspring = bp->k;
        Em = __ldcg(&b.sc[tl.img - 1].E);
        E0 = __ldcg(&sc.E);
        Ep = __ldcg(&b.sc[tl.img + 1].E);
    }
    const double tk = block_sum_records_wide<10, 4, RTHREADS, true>(
        b.row_part + (size_t)tl.img * b.rtpi * NPART, NPART, b.rtpi);
    __shared__ double s_d[10];
    if (threadIdx.x < 10) {
        sc.dots[threadIdx.x] = tk;
        s_d[threadIdx.x] = tk;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int ci = shard ? ci_ext : (climb ? climbing_image_warp(b, N, e0) : -1);
        if (threadIdx.x == 0) {
            if (tl.img == 1) bp->ci = ci;
            // mixed bands: 2 x 4e-6 energy units per atom, twice the bound
            // on the error of a step energy
            image_coef(b, tl.img, ci, s_d, Em, E0, Ep, kspring,
                       sizeof(T) == 4 ? 8e-6 * (double)b.n : 0.0);
        }
    }
}

// one block per image: sum the row-tile partials of the ten dots (spacings
// for the refinement check, outside the step)
__global__ void k_dots_reduce(const ImgRef *imgs, BandDev *bands) {
    ImgRef r = imgs[blockIdx.x];
    BandDev &b = bands[r.band];
    const double tk =
        block_sum_records<10, 12>(b.row_part + (size_t)r.img * b.rtpi * NPART, NPART, b.rtpi);
    if (threadIdx.x < 10) b.sc[r.img].dots[threadIdx.x] = tk;
}

// convergence test and FIRE decision on the band's parameters
__device__ inline void fire_logic(BandParams *bp, const double *tot) {
    bp->stale = 0;  // every image of the band has rebuilt its cell list
    const double P = tot[0], FF = tot[1], VV = tot[2];
    const double fmax_ = sqrt64(tot[3]);
    bp->P = P;
    bp->FF = FF;
    bp->VV = VV;
    bp->fmax = fmax_;
    if (!isfinite(P) || !isfinite(FF) || !isfinite(VV)) bp->status |= ST_NONFINITE;
    bp->converged = (bp->status == 0 && bp->ftol >= 0.0 && fmax_ < bp->ftol) ? 1 : 0;
    if (bp->status != 0 || bp->converged || bp->steps >= bp->move_limit) {
        bp->move = 0;
        bp->cv = 0.0;
        bp->cf = 0.0;
        return;
    }
    bp->move = 1;
    // FIRE (Bitzek et al. 2006): N_min 5, f_inc 1.1, f_dec 0.5, alpha0 0.1,
    // f_alpha 0.99; the first move after a reset skips the power test
    double cv = 1.0, cf = 0.0;
    if (!bp->fresh) {
        if (P > 0.0) {
            if (FF > 0.0) {
                cv = 1.0 - bp->alpha;
                cf = bp->alpha * sqrt64(VV) * rsqrt64(FF);
            }
            if (bp->npos > 5) {
                bp->dt = fmin(bp->dt * 1.1, bp->dt_max);
                bp->alpha *= 0.99;
            }
            bp->npos += 1;
        } else {
            cv = 0.0;
            cf = 0.0;
            bp->alpha = 0.1;
            bp->dt *= 0.5;
            bp->npos = 0;
        }
    }
    bp->fresh = 0;
    bp->cv = cv;
    bp->cf = cf;
    bp->steps += 1;
}

__device__ inline void atomic_max_nonneg(unsigned long long *bits, double v) {
    atomicMax(bits, (unsigned long long)__double_as_longlong(v));
}

// Pass 2: f_NEB rows (written for the state read-back and the move) and the
// largest row norm; the last tile of the band runs the convergence test and
// the FIRE decision on the sums of pass 1.
template <typename T>
__global__ void __launch_bounds__(RTHREADS, 4) k_neb_force(const Tile *tiles, BandDev *bands) {
    Tile tl = tiles[blockIdx.x];
    BandDev &b = bands[tl.band];
    // coefficients in T, converted once per block
    __shared__ T s_coef[2];
    if (threadIdx.x < 2) s_coef[threadIdx.x] = (T)b.sc[tl.img].coef[threadIdx.x];
    __syncthreads();
    const T ca = s_coef[0], cb = s_coef[1];
    const size_t stride = (size_t)b.rows * 3;
    const int r0 = tl.t * RTILE + RPT * (int)threadIdx.x;
    T mx = 0;
    if (r0 < b.rows) {
        const size_t o0 = tl.img * stride + (size_t)r0 * 3;
        T a[12], xp[12], xm[12], gv[12];
        ld12((const T *)b.X + o0, a);
        ld12((const T *)b.X + o0 + stride, xp);
        ld12((const T *)b.X + o0 - stride, xm);
        ld12((const T *)b.F + o0, gv);
#pragma unroll
        for (int c = 0; c < 12; ++c) gv[c] = gv[c] + ca * (xp[c] - a[c]) + cb * (a[c] - xm[c]);
        st12((T *)b.Fneb + o0, gv);
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const T ff = fma(gv[3 * q + 2], gv[3 * q + 2],
                             fma(gv[3 * q + 1], gv[3 * q + 1], gv[3 * q] * gv[3 * q]));
            mx = fmax(mx, ff);
        }
    }
    // block max of the row norms (a max is exact in any precision)
    __shared__ T smax[RTHREADS / 32];
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = mx;
    __syncthreads();
    BandParams *bp = b.bp;
    if (threadIdx.x == 0) {
        T m = (T)0;
        for (int q = 0; q < RTHREADS / 32; ++q) m = fmax(m, smax[q]);
        atomic_max_nonneg(&bp->fmax2_bits, (double)m);
    }
    if (!last_arrival(&bp->done_b, (unsigned)((bp->N - 2) * b.rtpi))) return;
    // the band's FIRE sums over the interior images, in image order (the
    // images' terms loaded in parallel, then added in order)
    __shared__ double s_tot[4];
    __shared__ double s_fire[3][64];
    const int N = bp->N;
    for (int base = 1; base < N - 1; base += 64) {
        const int cnt = min(64, N - 1 - base);
        if (threadIdx.x < 3 * cnt) {
            const int k = threadIdx.x / cnt, q = threadIdx.x % cnt;
            s_fire[k][q] = __ldcg(&b.sc[base + q].fire[k]);
        }
        __syncthreads();
        if (threadIdx.x < 3) {
            double v = base == 1 ? 0.0 : s_tot[threadIdx.x];
            for (int q = 0; q < cnt; ++q) v += s_fire[threadIdx.x][q];
            s_tot[threadIdx.x] = v;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        s_tot[3] = __longlong_as_double((long long)atomicExch(&bp->fmax2_bits, 0ull));
        if (bp->shard) {  // the caller combines the shards' sums
            bp->P = s_tot[0];
            bp->FF = s_tot[1];
            bp->VV = s_tot[2];
            bp->fmax = s_tot[3];
        } else {
            fire_logic(bp, s_tot);
        }
    }
}

// the FIRE decision of a shard on the sums of every shard of the band
__global__ void k_shard_fire(BandDev *band, double P, double FF, double VV, double fmax2) {
    const double tot[4] = {P, FF, VV, fmax2};
    fire_logic(band->bp, tot);
}

// One row of the move (Bitzek et al. 2006 with the band-global mixing
// cv, cf): v <- cv v + cf F_NEB; v += dt F_NEB; dX = dt v, scaled down to
// maxstep in norm; X += dX.  Atom rows and lattice rows take the same step.
template <typename T>
__device__ inline void fire_row(T *x, T *v, const T *fn, T cv, T cf, T dt, T ms) {
    T dx[3];
    T n2 = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        T vc = cv * v[c] + cf * fn[c];
        vc += dt * fn[c];
        v[c] = vc;
        dx[c] = dt * vc;
        n2 += dx[c] * dx[c];
    }
    if (n2 > ms * ms) {
        const T sc = ms / sqrt(n2);
#pragma unroll
        for (int c = 0; c < 3; ++c) dx[c] *= sc;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) x[c] += dx[c];
}

// The three lattice rows of one image, one warp: the move, then the new
// cell (image_cell_warp) and the bin vectors of the kept grid, so that the
// next evaluation's map-back finds them ready (cell_fresh) instead of
// starting its FP64 chain only then.  Runs beside the atom rows' blocks.
template <typename T>
__device__ inline void lattice_move_warp(const ImgRef r, BandDev *bands) {
    BandDev &b = bands[r.band];
    const BandParams *bp = b.bp;
    ImgScalars &sc = b.sc[r.img];
    const int lane = threadIdx.x & 31, l = lane % 9;
    // every load first (one round trip, under the row tiles' traffic)
    const int move = bp->move;
    const T cv = (T)bp->cv, cf = (T)bp->cf, dt = (T)bp->dt, ms = (T)bp->maxstep;
    const double skin = bp->skin;
    const CellIn k = cell_in(bp);
    const int nba = sc.nb[l / 3];
    float dbi[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) dbi[q] = lane == 0 ? sc.Dbif[q] : 0.0f;
    T x[3] = {0, 0, 0}, v[3] = {0, 0, 0}, fn[3] = {0, 0, 0};
    const size_t o = ((size_t)r.img * b.rows + b.n + (lane < 3 ? lane : 0)) * 3;
    if (lane < 3) {  // lane q moves lattice row n + q
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            x[c] = ((const T *)b.X)[o + c];
            v[c] = ((const T *)b.v)[o + c];
            fn[c] = ((const T *)b.Fneb)[o + c];
        }
    }
    if (!move) return;  // uniform over the warp
    if (lane < 3) {
        fire_row(x, v, fn, cv, cf, dt, ms);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ((T *)b.X)[o + c] = x[c];
            ((T *)b.v)[o + c] = v[c];
        }
    }
    // entry (l / 3, l % 3) of the moved lattice rows
    const T a0 = __shfl_sync(0xffffffffu, x[0], l / 3);
    const T a1 = __shfl_sync(0xffffffffu, x[1], l / 3);
    const T a2 = __shfl_sync(0xffffffffu, x[2], l / 3);
    const T xl = l % 3 == 0 ? a0 : (l % 3 == 1 ? a1 : a2);
    double h;
    const bool ok = image_cell_warp(k, (double)xl, sc, h);
    if (!ok && lane == 0) atomicOr(&b.bp->status, ST_NOT_SPD);
    __syncwarp();
    bin_vectors_warp(sc, nba, h);
    __syncwarp();
    if (lane == 0) {
        if (skin > 0.0) skin_terms(sc, dbi);  // for the next list decision
        sc.cell_fresh = 1;
    }
}

// Pass 3 on one row tile: the atom rows move, 4 rows a thread (lattice
// rows: lattice_move_warp; padding rows stay zero), and with a skin the
// tile records its largest displacement since the last list build.
template <typename T>
__device__ inline void move_tile(const Tile tl, BandDev *bands) {
    BandDev &b = bands[tl.band];
    const BandParams *bp = b.bp;
    // FIRE scalars in T, converted once per tile
    __shared__ T s_k[4];
    __shared__ int s_move;
    if (threadIdx.x == 0) {
        s_move = bp->move;
        s_k[0] = (T)bp->cv;
        s_k[1] = (T)bp->cf;
        s_k[2] = (T)bp->dt;
        s_k[3] = (T)bp->maxstep;
    }
    __syncthreads();
    if (!s_move) {  // uniform over the block
        __syncthreads();
        return;
    }
    const T cv = s_k[0], cf = s_k[1], dt = s_k[2], ms = s_k[3];
    const int r0 = tl.t * RTILE + RPT * (int)threadIdx.x;
    const int n = b.n;
    T d2 = 0;  // largest squared displacement of this thread's atom rows since the build
    if (r0 < n) {
        // rows r0 .. r0 + 3 lie within the padded stride (rows >= n + 3);
        // only atom rows move here (lattice rows: lattice_move_warp;
        // padding rows stay zero)
        const size_t o0 = (tl.img * (size_t)b.rows + (size_t)r0) * 3;
        T x[12], v[12], fn[12], rf[12];
        ld12((const T *)b.X + o0, x);
        ld12((const T *)b.v + o0, v);
        ld12((const T *)b.Fneb + o0, fn);
        if (b.ref_X) ld12((const T *)b.ref_X + o0, rf);  // with the others: one round trip
#pragma unroll
        for (int q = 0; q < RPT; ++q)
            if (r0 + q < n) fire_row(x + 3 * q, v + 3 * q, fn + 3 * q, cv, cf, dt, ms);
        if (r0 + RPT <= n) {
            st12((T *)b.v + o0, v);
            st12((T *)b.X + o0, x);
        } else {  // the last atom rows of the image: row by row
#pragma unroll
            for (int q = 0; q < RPT; ++q)
                if (r0 + q < n)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        ((T *)b.v)[o0 + 3 * q + c] = v[3 * q + c];
                        ((T *)b.X)[o0 + 3 * q + c] = x[3 * q + c];
                    }
        }
        if (b.ref_X) {
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                if (r0 + q < n) {
                    const T ex = x[3 * q] - rf[3 * q], ey = x[3 * q + 1] - rf[3 * q + 1],
                            ez = x[3 * q + 2] - rf[3 * q + 2];
                    d2 = fmax(d2, ex * ex + ey * ey + ez * ez);
                }
            }
        }
    }
    // the row tile's largest displacement for the next evaluation's list
    // decision (FP32, rounded up: the reuse test never sees one too small)
    if (b.ref_X) {
        __shared__ T wmax[RTHREADS / 32];
        for (int o = 16; o > 0; o >>= 1) d2 = fmax(d2, __shfl_xor_sync(0xffffffffu, d2, o));
        if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = d2;
        __syncthreads();
        if (threadIdx.x == 0) {
            T m = wmax[0];
            for (int q = 1; q < RTHREADS / 32; ++q) m = fmax(m, wmax[q]);
            b.skin_part[(size_t)tl.img * b.atpi + tl.t] = __fsqrt_ru(to_float_ru(m));
        }
    }
    __syncthreads();  // the shared scalars are reused by the block's next tile
}

// Pass 3: blocks 0 .. nimg-1 move the lattice rows of imgs[block] (one warp
// each, scheduled first so that their FP64 cell work overlaps the rest);
// every other block moves the atom rows of FU_TILES consecutive row tiles
// in turn (a grid that fits on the GPU at once: the tiles' loads are not
// split into a second wave that starts behind the first one's stores).
constexpr int FU_TILES = 2;
template <typename T>
__global__ void __launch_bounds__(RTHREADS, sizeof(T) == 4 ? 4 : 2)
    k_fire_update(const Tile *tiles, int ntiles, const ImgRef *imgs, int nimg, BandDev *bands) {
    if ((int)blockIdx.x < nimg) {
        if (threadIdx.x < 32) lattice_move_warp<T>(imgs[blockIdx.x], bands);
        return;
    }
    const int k0 = ((int)blockIdx.x - nimg) * FU_TILES;
    for (int k = k0; k < k0 + FU_TILES && k < ntiles; ++k) move_tile<T>(tiles[k], bands);
}

// X_img <- 1/2 (X_{img-1} + X_{img+1}) (image insertion; all rows)
template <typename T>
__global__ void k_midpoint(BandDev *band, int img) {
    BandDev &b = *band;
    const size_t stride = (size_t)b.rows * 3;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < stride;
         e += (size_t)gridDim.x * blockDim.x) {
        const T *xm = (const T *)b.X + (img - 1) * stride;
        const T *xp = (const T *)b.X + (img + 1) * stride;
        ((T *)b.X)[img * stride + e] = (T)0.5 * (xm[e] + xp[e]);
    }
}

// Band set-up (Sec. II.C and Sec. III): endpoints to generalised
// coordinates and linear interpolation.  s = R h^-1 for each endpoint; the
// final endpoint's s is shifted by whole lattice vectors to the periodic
// image nearest the initial one; R~ = s h0; lattice rows c B with
// B = D D^T, D = h0^-1 h (or c D).  With the filter off the final
// Cartesian positions are kept and the cell stays h0.  Image k gets
// X_0 + k/(N-1) (X_{N-1} - X_0), plus the caller's displacements on the
// interior atom rows.  Everything in FP64, stored as T.
template <typename T>
__global__ void k_setup(const double *R0, const double *R1, const double *noise, int N,
                        BandDev *band, const double *h1) {
    BandDev &b = *band;
    const BandParams *bp = b.bp;
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = b.n;
    if (row > n) return;
    const size_t stride = (size_t)b.rows * 3;
    double h1inv[9];
    inv3(h1, h1inv);
    if (row < n) {
        double s0[3], s1[3], a0[3], a1[3];
        for (int a = 0; a < 3; ++a) {
            s0[a] = R0[3 * row] * bp->h0inv[a] + R0[3 * row + 1] * bp->h0inv[3 + a] +
                    R0[3 * row + 2] * bp->h0inv[6 + a];
            s1[a] = R1[3 * row] * h1inv[a] + R1[3 * row + 1] * h1inv[3 + a] +
                    R1[3 * row + 2] * h1inv[6 + a];
            s1[a] -= rint(s1[a] - s0[a]);
        }
        const double *g1 = bp->filter ? bp->h0 : h1;
        for (int c = 0; c < 3; ++c) {
            a0[c] = s0[0] * bp->h0[c] + s0[1] * bp->h0[3 + c] + s0[2] * bp->h0[6 + c];
            a1[c] = s1[0] * g1[c] + s1[1] * g1[3 + c] + s1[2] * g1[6 + c];
        }
        for (int k = 0; k < N; ++k) {
            const double t = (double)k / (double)(N - 1);
            T *x = (T *)b.X + k * stride + (size_t)row * 3;
            for (int c = 0; c < 3; ++c) {
                double v = a0[c] + t * (a1[c] - a0[c]);
                if (noise && k > 0 && k < N - 1) v += noise[((size_t)(k - 1) * n + row) * 3 + c];
                x[c] = (T)v;
            }
        }
    } else {
        double D0[9], D1[9], L0[9], L1[9];
        matmul3(bp->h0inv, bp->h0, D0);
        matmul3(bp->h0inv, bp->filter ? h1 : bp->h0, D1);
        if (bp->variant == 0) {
            double t0[9], t1[9];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    t0[3 * i + j] = D0[3 * j + i];
                    t1[3 * i + j] = D1[3 * j + i];
                }
            matmul3(D0, t0, L0);
            matmul3(D1, t1, L1);
        } else {
            for (int k = 0; k < 9; ++k) { L0[k] = D0[k]; L1[k] = D1[k]; }
        }
        // stored relative to the reference cell, c (L - I): the rows keep
        // their precision in FP32 when the cell changes little along the
        // band (c = n makes c B large next to its differences)
        for (int k = 0; k < N; ++k) {
            const double t = (double)k / (double)(N - 1);
            T *x = (T *)b.X + k * stride + (size_t)n * 3;
            for (int e = 0; e < 9; ++e) {
                const double one = e % 4 == 0 ? 1.0 : 0.0;
                double a = bp->c * (L0[e] - one), c = bp->c * (L1[e] - one);
                x[e] = (T)(a + t * (c - a));
            }
        }
    }
}

// per band: moves, converged, status, fmax, climbing image, N (batch polling)
__global__ void k_gather_status(BandDev *bands, int nb, double *out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nb) return;
    const BandParams *bp = bands[k].bp;
    double *o = out + 6 * (size_t)k;
    o[0] = (double)bp->steps;
    o[1] = (double)bp->converged;
    o[2] = (double)bp->status;
    o[3] = bp->fmax;
    o[4] = (double)bp->ci;
    o[5] = (double)bp->N;
}

// ---- launchers -------------------------------------------------------------

void launch_gather_status(BandDev *bands, int nb, double *out, cudaStream_t s) {
    if (nb <= 0) return;
    k_gather_status<<<(nb + 127) / 128, 128, 0, s>>>(bands, nb, out);
}

template <typename T>
void launch_setup(const double *R0, const double *R1, const double *noise, int n, int N,
                  BandDev *band, cudaStream_t s, const double *h1) {
    k_setup<T><<<(n + 1 + 127) / 128, 128, 0, s>>>(R0, R1, noise, N, band, h1);
}

template <typename T>
void launch_image_finalize(const ImgRef *imgs, int count, BandDev *bands, cudaStream_t s) {
    if (count <= 0) return;
    k_image_finalize<T><<<count, FIN_THREADS, 0, s>>>(imgs, bands);
}
// pass 1 of the step (fused: per-image dots, NEB coefficients, FIRE sums)
template <typename T>
void launch_band_dots(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s) {
    if (ntiles <= 0) return;
    k_band_dots<T, true><<<ntiles, RTHREADS, 0, s>>>(tiles, bands);
}
// the dots alone (into the tile records; k_dots_reduce sums them per image)
template <typename T>
void launch_band_dots_only(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s) {
    if (ntiles <= 0) return;
    k_band_dots<T, false><<<ntiles, RTHREADS, 0, s>>>(tiles, bands);
}
void launch_dots_reduce(const ImgRef *imgs, int count, BandDev *bands, cudaStream_t s) {
    if (count <= 0) return;
    k_dots_reduce<<<count, RED_THREADS, 0, s>>>(imgs, bands);
}
void launch_shard_fire(BandDev *band, double P, double FF, double VV, double fmax2,
                       cudaStream_t s) {
    k_shard_fire<<<1, 1, 0, s>>>(band, P, FF, VV, fmax2);
}
template <typename T>
void launch_neb_force(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s) {
    if (ntiles <= 0) return;
    k_neb_force<T><<<ntiles, RTHREADS, 0, s>>>(tiles, bands);
}
template <typename T>
void launch_fire_update(const Tile *tiles, int ntiles, const ImgRef *imgs, int nimg,
                        BandDev *bands, cudaStream_t s) {
    if (ntiles + nimg <= 0) return;
    k_fire_update<T><<<nimg + (ntiles + FU_TILES - 1) / FU_TILES, RTHREADS, 0, s>>>(
        tiles, ntiles, imgs, nimg, bands);
}
template <typename T>
void launch_midpoint(BandDev *band, int img, int rows, cudaStream_t s) {
    int blocks = (rows * 3 + 255) / 256;
    blocks = blocks > 1024 ? 1024 : blocks;
    k_midpoint<T><<<blocks, 256, 0, s>>>(band, img);
}

#define CFNEB_INST(T)                                                                       \
    template void launch_image_finalize<T>(const ImgRef *, int, BandDev *, cudaStream_t);   \
    template void launch_band_dots<T>(const Tile *, int, BandDev *, cudaStream_t);          \
    template void launch_band_dots_only<T>(const Tile *, int, BandDev *, cudaStream_t);     \
    template void launch_neb_force<T>(const Tile *, int, BandDev *, cudaStream_t);          \
    template void launch_fire_update<T>(const Tile *, int, const ImgRef *, int, BandDev *,  \
                                        cudaStream_t);                                    \
    template void launch_midpoint<T>(BandDev *, int, int, cudaStream_t);                  \
    template void launch_setup<T>(const double *, const double *, const double *, int, int, \
                                  BandDev *, cudaStream_t, const double *);
CFNEB_INST(float)
CFNEB_INST(double)
#undef CFNEB_INST

}  // namespace cfneb
