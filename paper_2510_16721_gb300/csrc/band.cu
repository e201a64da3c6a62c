// Per-image reduction, cell-filter lattice force, NEB projection and FIRE.
//
// k_image_finalize  sums the force kernel's tile partials (FP64, slot order)
//                   into E and V, adds the external pressure (H = U + P Omega,
//                   V - P Omega I) and writes the three lattice rows of the
//                   generalised force: (1/c) 1/2 D^-T V_sym D^-1 for the
//                   rotation-free filter, (1/c) D^-T V for the deformation
//                   gradient (Sec. II.C).
// k_band_dots       per row tile: |dX+|^2, |dX-|^2, dX+.dX-, F.dX+, F.dX- in
//                   FP64 (dX+ = X_{i+1} - X_i, dX- = X_i - X_{i-1}).
// k_dots_reduce     sums those tile partials per image (one block per image).
// k_neb_coef        per band: climbing image, upwind tangent weights and the
//                   two coefficients with f_NEB = F + a dX+ + b dX-.  Since
//                   tau = w+ dX+ + w- dX-, |tau| and F.tau follow from the five
//                   dots, and the projection f - (f.t)t + k(|dX+|-|dX-|) t
//                   (Sec. II.A; climbing image f - 2 (f.t) t) becomes two
//                   scalars per image.
// k_neb_force       writes f_NEB and per-tile FIRE sums F.v, F.F, v.v and the
//                   largest row norm (fmax).
// k_fire_scalars    per band: convergence test, FIRE decision (Bitzek et al.
//                   2006, band-global power P = F.v) and the new dt, alpha.
// k_fire_update     v <- cv v + cf F; v += dt F; dX = dt v clamped per row to
//                   maxstep; X += dX (interior images only).
#include "common.cuh"

namespace cfneb {

template <typename T>
__global__ void k_image_finalize(const ImgRef *imgs, BandDev *bands) {
    ImgRef r = imgs[blockIdx.x];
    BandDev &b = bands[r.band];
    const BandParams *bp = b.bp;
    ImgScalars &sc = b.sc[r.img];
    // U, V (9), pairs, triples: tile partials summed in FP64, fixed order
    __shared__ double s_tot[12];
    const double tk =
        block_sum_records<12, 21>(b.atom_part + (size_t)r.img * b.atpi * NPART, NPART, b.atpi);
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

template <typename T>
__global__ void __launch_bounds__(TILE) k_band_dots(const Tile *tiles, BandDev *bands) {
    Tile tl = tiles[blockIdx.x];
    BandDev &b = bands[tl.band];
    T acc[5] = {0, 0, 0, 0, 0};
    const size_t stride = (size_t)b.rows * 3;
    const size_t o0 = tl.img * stride + ((size_t)tl.t * RTILE + threadIdx.x) * 3;
    const T *__restrict__ X0 = (const T *)b.X + o0;
    const T *__restrict__ F0 = (const T *)b.F + o0;
    const int nrow = b.rows - tl.t * RTILE - (int)threadIdx.x;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        if (k * TILE < nrow) {
            const T *x0 = X0 + k * TILE * 3, *f = F0 + k * TILE * 3;
            for (int c = 0; c < 3; ++c) {
                const T a = x0[c];
                const T dp = x0[stride + c] - a, dm = a - x0[c - (long long)stride], fc = f[c];
                acc[0] += dp * dp;
                acc[1] += dm * dm;
                acc[2] += dp * dm;
                acc[3] += fc * dp;
                acc[4] += fc * dm;
            }
        }
    }
    block_sum_store<5, T>(acc, b.row_part + ((size_t)tl.img * b.rtpi + tl.t) * NPART);
}

// one block per image: sum the row-tile partials of the five dots
__global__ void k_dots_reduce(const ImgRef *imgs, BandDev *bands) {
    ImgRef r = imgs[blockIdx.x];
    BandDev &b = bands[r.band];
    const double tk =
        block_sum_records<5, 16>(b.row_part + (size_t)r.img * b.rtpi * NPART, NPART, b.rtpi);
    if (threadIdx.x < 5) b.sc[r.img].dots[threadIdx.x] = tk;
}

// one block (one thread per image) per band
__global__ void k_neb_coef(const int *band_ids, BandDev *bands) {
    BandDev &b = bands[band_ids[blockIdx.x]];
    BandParams *bp = b.bp;
    const int N = bp->N;
    __shared__ int s_ci;
    if (threadIdx.x == 0) {
        int ci = -1;
        if (bp->climb) {
            double best = 0.0;
            for (int i = 1; i < N - 1; ++i)
                if (ci < 0 || b.sc[i].E > best) {
                    best = b.sc[i].E;
                    ci = i;
                }
        }
        s_ci = ci;
        bp->ci = ci;
    }
    __syncthreads();
    for (int i = 1 + threadIdx.x; i < N - 1; i += blockDim.x) {
        const ImgScalars &sc = b.sc[i];
        const double Em = b.sc[i - 1].E, E0 = sc.E, Ep = b.sc[i + 1].E;
        double wp, wm;
        if (Ep > E0 && E0 > Em) {
            wp = 1.0; wm = 0.0;
        } else if (Ep < E0 && E0 < Em) {
            wp = 0.0; wm = 1.0;
        } else {
            const double a = fabs(Ep - E0), c = fabs(Em - E0);
            const double dmax = fmax(a, c), dmin = fmin(a, c);
            if (dmax == 0.0) {
                wp = 1.0; wm = 1.0;
            } else if (Ep > Em) {
                wp = dmax; wm = dmin;
            } else {
                wp = dmin; wm = dmax;
            }
        }
        const double pp = sc.dots[0], mm = sc.dots[1], pm = sc.dots[2];
        const double fp = sc.dots[3], fm = sc.dots[4];
        const double tt = wp * wp * pp + 2.0 * wp * wm * pm + wm * wm * mm;
        const double tn = sqrt(tt);
        const double ft = (wp * fp + wm * fm) / tn;  // F . tau_hat
        double gamma;
        if (i == s_ci) {
            gamma = -2.0 * ft;
        } else {
            gamma = bp->k * (sqrt(pp) - sqrt(mm)) - ft;
        }
        b.sc[i].coef[0] = gamma * wp / tn;
        b.sc[i].coef[1] = gamma * wm / tn;
    }
}

template <typename T>
__global__ void __launch_bounds__(TILE) k_neb_force(const Tile *tiles, BandDev *bands) {
    Tile tl = tiles[blockIdx.x];
    BandDev &b = bands[tl.band];
    T acc[4] = {0, 0, 0, 0};  // F.v, F.F, v.v, largest row |F|^2 (fmax)
    // coefficients in T, converted once per block
    __shared__ T s_coef[2];
    if (threadIdx.x < 2) s_coef[threadIdx.x] = (T)b.sc[tl.img].coef[threadIdx.x];
    __syncthreads();
    const T ca = s_coef[0], cb = s_coef[1];
    const size_t stride = (size_t)b.rows * 3;
    const size_t o0 = tl.img * stride + ((size_t)tl.t * RTILE + threadIdx.x) * 3;
    const T *__restrict__ X0 = (const T *)b.X + o0;
    const T *__restrict__ F0 = (const T *)b.F + o0;
    const T *__restrict__ V0 = (const T *)b.v + o0;
    T *__restrict__ G0 = (T *)b.Fneb + o0;
    const int nrow = b.rows - tl.t * RTILE - (int)threadIdx.x;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        if (k * TILE < nrow) {
            const size_t q = (size_t)k * TILE * 3;
            T ff = 0;
            for (int c = 0; c < 3; ++c) {
                const T a = X0[q + c];
                const T g = F0[q + c] + ca * (X0[q + stride + c] - a) +
                            cb * (a - X0[q + c - stride]);
                const T vc = V0[q + c];
                G0[q + c] = g;
                acc[0] += g * vc;
                ff += g * g;
                acc[2] += vc * vc;
            }
            acc[1] += ff;
            acc[3] = fmax(acc[3], ff);
        }
    }
    T three[3] = {acc[0], acc[1], acc[2]};
    double *part = b.row_part + ((size_t)tl.img * b.rtpi + tl.t) * NPART;
    block_sum_store<3, T>(three, part + 5);
    // block max of the row norms, in T (a max is exact in any precision)
    __shared__ T smax[TILE / 32];
    T m = acc[3];
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        T mx = (T)0;
        for (int q = 0; q < TILE / 32; ++q) mx = fmax(mx, smax[q]);
        part[8] = (double)mx;
    }
}

// one block per band; the threads sum the tile partials of every interior
// image, thread 0 runs the FIRE logic
// convergence test and FIRE decision on the band's parameters
__device__ inline void fire_logic(BandParams *bp, const double *tot) {
    bp->stale = 0;  // every image of the band has rebuilt its cell list
    const double P = tot[0], FF = tot[1], VV = tot[2];
    const double fmax_ = sqrt(tot[3]);
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
                cf = bp->alpha * sqrt(VV) / sqrt(FF);
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

__global__ void k_fire_scalars(const int *band_ids, BandDev *bands) {
    BandDev &b = bands[band_ids[blockIdx.x]];
    // the band's parameters are staged in shared memory, updated by thread 0
    // and written back (no other kernel touches them meanwhile)
    __shared__ BandParams s_bp;
    stage_copy(&s_bp, b.bp);
    __syncthreads();
    const int N = s_bp.N;
    // the row-tile partials of images 1..N-2, one fixed strided subset per
    // thread, then a fixed-order block sum
    const int nt = (N - 2) * b.rtpi;
    const double *part0 = b.row_part + (size_t)b.rtpi * NPART;
    // F.v, F.F, v.v summed, the largest row |F|^2 taken, each over 32 fixed
    // strided subsets and then in subset order (few FP64 instructions)
    constexpr int G = 32;
    __shared__ double s_part[G * 4], s_tot[4];
    if (threadIdx.x < 4 * G) {
        const int k = threadIdx.x % 4, g = threadIdx.x / 4;
        double v = 0.0;
#pragma unroll 8
        for (int q = g; q < nt; q += G) {
            const double x = part0[(size_t)q * NPART + 5 + k];
            v = k == 3 ? fmax(v, x) : v + x;
        }
        s_part[g * 4 + k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        const int k = threadIdx.x;
        double v = 0.0;
        for (int g = 0; g < G; ++g) v = k == 3 ? fmax(v, s_part[g * 4 + k]) : v + s_part[g * 4 + k];
        s_tot[k] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) fire_logic(&s_bp, s_tot);
    __syncthreads();
    stage_copy(b.bp, &s_bp);
}

template <typename T>
__global__ void __launch_bounds__(TILE) k_fire_update(const Tile *tiles, BandDev *bands) {
    Tile tl = tiles[blockIdx.x];
    BandDev &b = bands[tl.band];
    const BandParams *bp = b.bp;
    if (!bp->move) return;  // uniform over the block
    // FIRE scalars in T, converted once per block
    __shared__ T s_k[4];
    if (threadIdx.x == 0) {
        s_k[0] = (T)bp->cv;
        s_k[1] = (T)bp->cf;
        s_k[2] = (T)bp->dt;
        s_k[3] = (T)bp->maxstep;
    }
    __syncthreads();
    const T cv = s_k[0], cf = s_k[1], dt = s_k[2], ms = s_k[3];
    const size_t o0 = (tl.img * (size_t)b.rows + (size_t)tl.t * RTILE + threadIdx.x) * 3;
    T *__restrict__ X = (T *)b.X + o0;
    T *__restrict__ V = (T *)b.v + o0;
    const T *__restrict__ Fn = (const T *)b.Fneb + o0;
    const int nrow = b.rows - tl.t * RTILE - (int)threadIdx.x;  // rows k * TILE < nrow exist
    // all loads first (rows of one thread are TILE apart: independent)
    T xr[RPT][3], vr[RPT][3], fr[RPT][3];
#pragma unroll
    for (int k = 0; k < RPT; ++k)
        if (k * TILE < nrow)
            for (int c = 0; c < 3; ++c) {
                xr[k][c] = X[k * TILE * 3 + c];
                vr[k][c] = V[k * TILE * 3 + c];
                fr[k][c] = Fn[k * TILE * 3 + c];
            }
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        if (k * TILE >= nrow) break;
        T dx[3];
        T n2 = 0;
        for (int c = 0; c < 3; ++c) {
            T vc = cv * vr[k][c] + cf * fr[k][c];
            vc += dt * fr[k][c];
            V[k * TILE * 3 + c] = vc;
            dx[c] = dt * vc;
            n2 += dx[c] * dx[c];
        }
        if (n2 > ms * ms) {
            const T s = ms / sqrt(n2);
            for (int c = 0; c < 3; ++c) dx[c] *= s;
        }
        for (int c = 0; c < 3; ++c) X[k * TILE * 3 + c] = xr[k][c] + dx[c];
    }
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
        for (int k = 0; k < N; ++k) {
            const double t = (double)k / (double)(N - 1);
            T *x = (T *)b.X + k * stride + (size_t)n * 3;
            for (int e = 0; e < 9; ++e) {
                double a = bp->c * L0[e], c = bp->c * L1[e];
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
    k_image_finalize<T><<<count, RED_THREADS, 0, s>>>(imgs, bands);
}
template <typename T>
void launch_band_dots(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s) {
    if (ntiles <= 0) return;
    k_band_dots<T><<<ntiles, TILE, 0, s>>>(tiles, bands);
}
void launch_dots_reduce(const ImgRef *imgs, int count, BandDev *bands, cudaStream_t s) {
    if (count <= 0) return;
    k_dots_reduce<<<count, RED_THREADS, 0, s>>>(imgs, bands);
}
void launch_neb_coef(const int *band_ids, int nbands, BandDev *bands, cudaStream_t s) {
    if (nbands <= 0) return;
    k_neb_coef<<<nbands, 32, 0, s>>>(band_ids, bands);
}
template <typename T>
void launch_neb_force(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s) {
    if (ntiles <= 0) return;
    k_neb_force<T><<<ntiles, TILE, 0, s>>>(tiles, bands);
}
void launch_fire_scalars(const int *band_ids, int nbands, BandDev *bands, cudaStream_t s) {
    if (nbands <= 0) return;
    k_fire_scalars<<<nbands, 1024, 0, s>>>(band_ids, bands);
}
template <typename T>
void launch_fire_update(const Tile *tiles, int ntiles, BandDev *bands, cudaStream_t s) {
    if (ntiles <= 0) return;
    k_fire_update<T><<<ntiles, TILE, 0, s>>>(tiles, bands);
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
    template void launch_neb_force<T>(const Tile *, int, BandDev *, cudaStream_t);          \
    template void launch_fire_update<T>(const Tile *, int, BandDev *, cudaStream_t);        \
    template void launch_midpoint<T>(BandDev *, int, int, cudaStream_t);                  \
    template void launch_setup<T>(const double *, const double *, const double *, int, int, \
                                  BandDev *, cudaStream_t, const double *);
CFNEB_INST(float)
CFNEB_INST(double)
#undef CFNEB_INST

}  // namespace cfneb
