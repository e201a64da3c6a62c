// Host side of the CFNEB library: band allocation, tile tables, step
// enqueueing (direct launches or a captured CUDA graph), refinement and the
// C ABI of include/cfneb.h.
//
// The host only allocates, builds launch tables, orders streams and moves
// data; every arithmetic step of the method (set-up mapping, interpolation,
// map-back, cell list, forces, cell filter, NEB projection, FIRE, midpoint
// insertion) runs in the kernels of this library.  Refinement decisions
// (which segment to split, which image to drop) are made on the host from
// spacings and energies the kernels computed, because they change the launch
// shape.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/cfneb.h"
#include "common.cuh"

using namespace cfneb;

namespace {

thread_local std::string g_last_error;

struct CudaFail {
    cudaError_t e;
};

#define CK(x)                                                                            \
    do {                                                                                 \
        cudaError_t _e = (x);                                                            \
        if (_e != cudaSuccess) {                                                         \
            g_last_error = std::string(#x) + ": " + cudaGetErrorString(_e);              \
            throw CudaFail{_e};                                                          \
        }                                                                                \
    } while (0)

enum KernelId {
    K_MAPBACK, K_BIN_ASSIGN, K_BIN_TILESUM, K_BIN_TILESCAN, K_BIN_SCANFILL, K_BIN_SCATTER,
    K_BIN_ORDER, K_LJ, K_TERS_PARTIALS, K_TERS_GATHER, K_IMAGE_FINALIZE, K_BAND_DOTS,
    K_DOTS_REDUCE, K_NEB_COEF, K_NEB_FORCE, K_FIRE_SCALARS, K_FIRE_UPDATE, K_COUNT
};
const char *kKernelNames[K_COUNT] = {
    "mapback", "bin_assign", "bin_tilesum", "bin_tilescan", "bin_scanfill", "bin_scatter",
    "bin_order", "lj_force", "tersoff_partials", "tersoff_gather", "image_finalize",
    "band_dots", "dots_reduce", "neb_coef", "neb_force", "fire_scalars", "fire_update"};

const double kTersoff1988C[11] = {1393.6, 346.74, 3.4879, 2.2119, 1.5724e-7, 0.72751,
                                  38049.0, 4.3484, -0.57058, 1.95, 0.15};

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace

// One band: its device buffers and host-side configuration.
struct cfneb_band {
    int n = 0, N = 0, ncap = 0, precision = 0, kind = 0;
    size_t ts = 8;               // sizeof(T)
    cfneb_options opt{};
    cfneb_cell_filter filt{};
    double h0[9]{}, c = 1.0;
    BandDev dv{};                // host copy holding device pointers
    BandDev *d_self = nullptr;   // device copy (array of one)
    std::vector<void *> allocs;
    size_t bytes = 0;
    long long last_change = 0;
    long long last_check = -1;
    double ftol = -1.0;
    // stream ordering
    cudaStream_t user = nullptr, s = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // launch tables (device) and their sizes
    Tile *d_atiles = nullptr;    // atom tiles of the interior images
    Tile *d_rtiles = nullptr;    // row tiles of the interior images
    ImgRef *d_imgs = nullptr;    // interior images
    int *d_band_ids = nullptr;
    Tile *d_scratch_tiles = nullptr;   // tables for ad-hoc image sets
    ImgRef *d_scratch_imgs = nullptr;
    int n_atiles = 0, n_rtiles = 0, n_imgs = 0;
    // graph
    cudaGraphExec_t gexec = nullptr;
    bool graph_dirty = true;
    // profiling
    bool prof = false;
    double prof_ms[K_COUNT]{};
    long long prof_n[K_COUNT]{};
    std::vector<cudaEvent_t> prof_ev;
    // pinned host mirror of BandParams
    BandParams *h_bp = nullptr;
};

namespace {

void *dalloc(cfneb_band *b, size_t bytes) {
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        g_last_error = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        throw CudaFail{e};
    }
    b->allocs.push_back(p);
    b->bytes += bytes;
    return p;
}

void free_band(cfneb_band *b) {
    if (!b) return;
    if (b->s) cudaStreamSynchronize(b->s);
    for (void *p : b->allocs) cudaFree(p);
    b->allocs.clear();
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    for (auto e : b->prof_ev) cudaEventDestroy(e);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->s) cudaStreamDestroy(b->s);
    if (b->h_bp) cudaFreeHost(b->h_bp);
    delete b;
}

// perpendicular widths of a cell (rows = lattice vectors)
void widths(const double *h, double *w) {
    double vol = std::fabs(det3(h));
    for (int a = 0; a < 3; ++a) {
        const double *u = h + 3 * ((a + 1) % 3), *v = h + 3 * ((a + 2) % 3);
        double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2],
               cz = u[0] * v[1] - u[1] * v[0];
        w[a] = vol / std::sqrt(cx * cx + cy * cy + cz * cz);
    }
}

int bins_for(const double *h, double bw) {
    double w[3];
    widths(h, w);
    long long p = 1;
    for (int a = 0; a < 3; ++a) p *= std::max(1, (int)std::floor(w[a] / bw));
    return (int)std::min<long long>(p, 1LL << 26);
}

// stream ordering with the caller's stream
void enter(cfneb_band *b) {
    CK(cudaEventRecord(b->ev_in, b->user));
    CK(cudaStreamWaitEvent(b->s, b->ev_in, 0));
}
void leave(cfneb_band *b) {
    CK(cudaEventRecord(b->ev_out, b->s));
    CK(cudaStreamWaitEvent(b->user, b->ev_out, 0));
}

// ---- launch tables -------------------------------------------------------

void build_tables(cfneb_band *b) {
    std::vector<Tile> at, rt;
    std::vector<ImgRef> im;
    for (int i = 1; i < b->N - 1; ++i) {
        im.push_back({0, i});
        for (int t = 0; t < b->dv.atpi; ++t) at.push_back({0, i, t, 0});
        for (int t = 0; t < b->dv.rtpi; ++t) rt.push_back({0, i, t, 0});
    }
    b->n_atiles = (int)at.size();
    b->n_rtiles = (int)rt.size();
    b->n_imgs = (int)im.size();
    if (!at.empty())
        CK(cudaMemcpyAsync(b->d_atiles, at.data(), at.size() * sizeof(Tile),
                           cudaMemcpyHostToDevice, b->s));
    if (!rt.empty())
        CK(cudaMemcpyAsync(b->d_rtiles, rt.data(), rt.size() * sizeof(Tile),
                           cudaMemcpyHostToDevice, b->s));
    if (!im.empty())
        CK(cudaMemcpyAsync(b->d_imgs, im.data(), im.size() * sizeof(ImgRef),
                           cudaMemcpyHostToDevice, b->s));
    CK(cudaStreamSynchronize(b->s));  // host vectors go out of scope
    b->graph_dirty = true;
}

// ---- kernel sequences ------------------------------------------------------

struct Launcher {
    cfneb_band *b;
    int k = 0;
    void pre(int id) {
        if (b->prof) CK(cudaEventRecord(b->prof_ev[2 * k], b->s));
        (void)id;
    }
    void post(int id) {
        if (b->prof) {
            CK(cudaEventRecord(b->prof_ev[2 * k + 1], b->s));
            ids.push_back(id);
            ++k;
        }
    }
    std::vector<int> ids;
};

template <typename T>
void enqueue_eval(cfneb_band *b, Launcher &L, const ImgRef *imgs, int nimg, const Tile *atiles,
                  int natiles, bool forces = true) {
    BandDev *d = b->d_self;
    cudaStream_t s = b->s;
    L.pre(K_MAPBACK); launch_mapback<T>(imgs, nimg, d, s); L.post(K_MAPBACK);
    L.pre(K_BIN_ASSIGN); launch_bin_assign<T>(atiles, natiles, d, s); L.post(K_BIN_ASSIGN);
    const int nbc = b->dv.nbins_cap;
    L.pre(K_BIN_TILESUM); launch_bin_scan(imgs, nimg, nbc, d, s, 0); L.post(K_BIN_TILESUM);
    L.pre(K_BIN_TILESCAN); launch_bin_scan(imgs, nimg, nbc, d, s, 1); L.post(K_BIN_TILESCAN);
    L.pre(K_BIN_SCANFILL); launch_bin_scan(imgs, nimg, nbc, d, s, 2); L.post(K_BIN_SCANFILL);
    L.pre(K_BIN_SCATTER); launch_bin_scatter(atiles, natiles, d, s); L.post(K_BIN_SCATTER);
    L.pre(K_BIN_ORDER); launch_bin_order<T>(imgs, nimg, b->dv.nbins_cap, d, s); L.post(K_BIN_ORDER);
    if (!forces) {
        launch_energy64<T>(atiles, natiles, imgs, nimg, d, s);
        return;
    }
    if (b->kind == CFNEB_LJ) {
        L.pre(K_LJ); launch_lj<T>(atiles, natiles, d, s); L.post(K_LJ);
    } else {
        L.pre(K_TERS_PARTIALS); launch_tersoff_partials<T>(atiles, natiles, d, s);
        L.post(K_TERS_PARTIALS);
        L.pre(K_TERS_GATHER); launch_tersoff_gather<T>(atiles, natiles, d, s);
        L.post(K_TERS_GATHER);
    }
    L.pre(K_IMAGE_FINALIZE); launch_image_finalize<T>(imgs, nimg, d, s); L.post(K_IMAGE_FINALIZE);
}

template <typename T>
void enqueue_step(cfneb_band *b, Launcher &L) {
    BandDev *d = b->d_self;
    cudaStream_t s = b->s;
    enqueue_eval<T>(b, L, b->d_imgs, b->n_imgs, b->d_atiles, b->n_atiles);
    L.pre(K_BAND_DOTS); launch_band_dots<T>(b->d_rtiles, b->n_rtiles, d, s); L.post(K_BAND_DOTS);
    L.pre(K_DOTS_REDUCE); launch_dots_reduce(b->d_imgs, b->n_imgs, d, s); L.post(K_DOTS_REDUCE);
    L.pre(K_NEB_COEF); launch_neb_coef(b->d_band_ids, 1, d, s); L.post(K_NEB_COEF);
    L.pre(K_NEB_FORCE); launch_neb_force<T>(b->d_rtiles, b->n_rtiles, d, s); L.post(K_NEB_FORCE);
    L.pre(K_FIRE_SCALARS); launch_fire_scalars(b->d_band_ids, 1, d, s); L.post(K_FIRE_SCALARS);
    L.pre(K_FIRE_UPDATE); launch_fire_update<T>(b->d_rtiles, b->n_rtiles, d, s);
    L.post(K_FIRE_UPDATE);
}

int launches_per_step(const cfneb_band *b) {
    return 7 + (b->kind == CFNEB_LJ ? 1 : 2) + 1 + 6;
}

void run_step_sequence(cfneb_band *b) {
    Launcher L{b};
    if (b->precision == CFNEB_MIXED) enqueue_step<float>(b, L);
    else enqueue_step<double>(b, L);
    CK(cudaGetLastError());
    if (b->prof) {
        CK(cudaStreamSynchronize(b->s));
        for (int q = 0; q < L.k; ++q) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, b->prof_ev[2 * q], b->prof_ev[2 * q + 1]));
            b->prof_ms[L.ids[q]] += ms;
            b->prof_n[L.ids[q]] += 1;
        }
    }
}

void capture_graph(cfneb_band *b) {
    if (b->gexec) {
        CK(cudaGraphExecDestroy(b->gexec));
        b->gexec = nullptr;
    }
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal));
    Launcher L{b};
    try {
        if (b->precision == CFNEB_MIXED) enqueue_step<float>(b, L);
        else enqueue_step<double>(b, L);
    } catch (...) {
        cudaStreamEndCapture(b->s, &g);
        if (g) cudaGraphDestroy(g);
        throw;
    }
    CK(cudaStreamEndCapture(b->s, &g));
    cudaError_t e = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    CK(e);
    b->graph_dirty = false;
}

void steps(cfneb_band *b, int n) {
    if (n <= 0 || b->N < 3) return;
    if (b->prof) {
        for (int i = 0; i < n; ++i) run_step_sequence(b);
        return;
    }
    if (b->graph_dirty || !b->gexec) capture_graph(b);
    for (int i = 0; i < n; ++i) CK(cudaGraphLaunch(b->gexec, b->s));
}

// evaluate an arbitrary list of images of the band (endpoints, new images)
void eval_images(cfneb_band *b, const std::vector<int> &imgs) {
    std::vector<ImgRef> im;
    std::vector<Tile> at;
    for (int i : imgs) {
        im.push_back({0, i});
        for (int t = 0; t < b->dv.atpi; ++t) at.push_back({0, i, t, 0});
    }
    CK(cudaMemcpyAsync(b->d_scratch_imgs, im.data(), im.size() * sizeof(ImgRef),
                       cudaMemcpyHostToDevice, b->s));
    CK(cudaMemcpyAsync(b->d_scratch_tiles, at.data(), at.size() * sizeof(Tile),
                       cudaMemcpyHostToDevice, b->s));
    Launcher L{b};
    bool prof = b->prof;
    b->prof = false;
    if (b->precision == CFNEB_MIXED)
        enqueue_eval<float>(b, L, b->d_scratch_imgs, (int)im.size(), b->d_scratch_tiles,
                            (int)at.size());
    else
        enqueue_eval<double>(b, L, b->d_scratch_imgs, (int)im.size(), b->d_scratch_tiles,
                             (int)at.size());
    b->prof = prof;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(b->s));
}

// FP64 energies (ImgScalars::E64) of the images' current coordinates:
// map-back, cell list and the FP64 energy kernel, no forces
void refine_energies(cfneb_band *b, int first, int count) {
    std::vector<ImgRef> im;
    std::vector<Tile> at;
    for (int i = first; i < first + count; ++i) {
        im.push_back({0, i});
        for (int t = 0; t < b->dv.atpi; ++t) at.push_back({0, i, t, 0});
    }
    CK(cudaMemcpyAsync(b->d_scratch_imgs, im.data(), im.size() * sizeof(ImgRef),
                       cudaMemcpyHostToDevice, b->s));
    CK(cudaMemcpyAsync(b->d_scratch_tiles, at.data(), at.size() * sizeof(Tile),
                       cudaMemcpyHostToDevice, b->s));
    Launcher L{b};
    bool prof = b->prof;
    b->prof = false;
    if (b->precision == CFNEB_MIXED)
        enqueue_eval<float>(b, L, b->d_scratch_imgs, (int)im.size(), b->d_scratch_tiles,
                            (int)at.size(), false);
    else
        enqueue_eval<double>(b, L, b->d_scratch_imgs, (int)im.size(), b->d_scratch_tiles,
                             (int)at.size(), false);
    b->prof = prof;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(b->s));
}

void read_params(cfneb_band *b) {
    CK(cudaMemcpyAsync(b->h_bp, b->dv.bp, sizeof(BandParams), cudaMemcpyDeviceToHost, b->s));
    CK(cudaStreamSynchronize(b->s));
}

int status_from_bits(int bits) {
    if (bits & ST_NONFINITE) return CFNEB_ERR_NONFINITE;
    if (bits & ST_NOT_SPD) return CFNEB_ERR_NOT_SPD;
    if (bits & ST_NBR_OVERFLOW) return CFNEB_ERR_NBR_OVERFLOW;
    return CFNEB_OK;
}

// write FIRE reset values into the device params and zero velocities
void fire_reset(cfneb_band *b) {
    read_params(b);
    BandParams *p = b->h_bp;
    p->dt = p->dt0;
    p->alpha = 0.1;
    p->npos = 0;
    p->fresh = 1;
    CK(cudaMemcpyAsync(b->dv.bp, p, sizeof(BandParams), cudaMemcpyHostToDevice, b->s));
    CK(cudaMemsetAsync(b->dv.v, 0, (size_t)b->ncap * b->dv.rows * 3 * b->ts, b->s));
    CK(cudaStreamSynchronize(b->s));
}

void set_N(cfneb_band *b, int N) {
    b->N = N;
    read_params(b);
    b->h_bp->N = N;
    CK(cudaMemcpyAsync(b->dv.bp, b->h_bp, sizeof(BandParams), cudaMemcpyHostToDevice, b->s));
    CK(cudaStreamSynchronize(b->s));
    build_tables(b);
}

// move images [from, N) by `delta` slots (+1: open a gap, -1: close one)
void shift_images(cfneb_band *b, int from, int delta) {
    const size_t vec = (size_t)b->dv.rows * 3 * b->ts;
    auto mv = [&](void *base, size_t each) {
        char *p = (char *)base;
        if (delta > 0) {
            for (int i = b->N - 1; i >= from; --i)
                CK(cudaMemcpyAsync(p + (i + 1) * each, p + i * each, each,
                                   cudaMemcpyDeviceToDevice, b->s));
        } else {
            for (int i = from; i < b->N; ++i)
                CK(cudaMemcpyAsync(p + (i - 1) * each, p + i * each, each,
                                   cudaMemcpyDeviceToDevice, b->s));
        }
    };
    mv(b->dv.X, vec);
    mv(b->dv.F, vec);
    mv(b->dv.Fneb, vec);
    mv(b->dv.sc, sizeof(ImgScalars));
}

int insert_image(cfneb_band *b, int after) {
    if (after < 0 || after >= b->N - 1) return CFNEB_ERR_INVALID_ARG;
    if (b->N >= b->ncap) return CFNEB_ERR_STATE;
    shift_images(b, after + 1, +1);
    // image after+1 is now the gap between after and after+2
    if (b->precision == CFNEB_MIXED) launch_midpoint<float>(b->d_self, after + 1, b->dv.rows, b->s);
    else launch_midpoint<double>(b->d_self, after + 1, b->dv.rows, b->s);
    CK(cudaGetLastError());
    set_N(b, b->N + 1);
    fire_reset(b);
    return CFNEB_OK;
}

int delete_image(cfneb_band *b, int index) {
    if (index <= 0 || index >= b->N - 1) return CFNEB_ERR_INVALID_ARG;
    if (b->N <= 3 || b->N <= b->opt.n_min) return CFNEB_ERR_STATE;
    shift_images(b, index + 1, -1);
    set_N(b, b->N - 1);
    fire_reset(b);
    return CFNEB_OK;
}

// spacings l_s = |X_{s+1} - X_s| of the current X (after the last move):
// the band-dot kernels over every image but the last give |dX+|^2.
void spacings(cfneb_band *b, std::vector<double> &ell) {
    std::vector<Tile> rt;
    std::vector<ImgRef> im;
    for (int i = 0; i < b->N - 1; ++i) {
        im.push_back({0, i});
        for (int t = 0; t < b->dv.rtpi; ++t) rt.push_back({0, i, t, 0});
    }
    // the dot kernel reads X_{i-1} and X_{i+1}: run it on images 1..N-2 only;
    // image 1's |dX-| is the first segment
    CK(cudaMemcpyAsync(b->d_scratch_imgs, im.data(), im.size() * sizeof(ImgRef),
                       cudaMemcpyHostToDevice, b->s));
    CK(cudaMemcpyAsync(b->d_scratch_tiles, rt.data(), rt.size() * sizeof(Tile),
                       cudaMemcpyHostToDevice, b->s));
    if (b->precision == CFNEB_MIXED)
        launch_band_dots<float>(b->d_scratch_tiles + b->dv.rtpi, (int)rt.size() - b->dv.rtpi,
                                b->d_self, b->s);
    else
        launch_band_dots<double>(b->d_scratch_tiles + b->dv.rtpi, (int)rt.size() - b->dv.rtpi,
                                 b->d_self, b->s);
    launch_dots_reduce(b->d_scratch_imgs + 1, (int)im.size() - 1, b->d_self, b->s);
    CK(cudaGetLastError());
    std::vector<ImgScalars> sc(b->N);
    CK(cudaMemcpyAsync(sc.data(), b->dv.sc, b->N * sizeof(ImgScalars), cudaMemcpyDeviceToHost,
                       b->s));
    CK(cudaStreamSynchronize(b->s));
    ell.assign(b->N - 1, 0.0);
    ell[0] = std::sqrt(sc[1].dots[1]);            // |X_1 - X_0|
    for (int i = 1; i < b->N - 1; ++i) ell[i] = std::sqrt(sc[i].dots[0]);  // |X_{i+1} - X_i|
}

// one refinement check with the rules of the oracle (spacing based)
void refine(cfneb_band *b) {
    std::vector<double> ell;
    spacings(b, ell);
    double mean = 0.0;
    for (double l : ell) mean += l;
    mean /= (double)ell.size();
    int s = 0;
    for (int i = 1; i < (int)ell.size(); ++i)
        if (ell[i] > ell[s]) s = i;
    read_params(b);
    long long steps_now = b->h_bp->steps;
    int ci = b->h_bp->ci;
    if (ell[s] > b->opt.alpha_ins * mean && b->N < b->opt.n_max) {
        insert_image(b, s);
        b->last_change = steps_now;
        return;
    }
    if (b->N > b->opt.n_min) {
        int best_j = -1;
        double best = 0.0;
        for (int j = 1; j < b->N - 1; ++j) {
            if (b->opt.climb && j == ci) continue;
            double pair = ell[j - 1] + ell[j];
            if (best_j < 0 || pair < best) {
                best = pair;
                best_j = j;
            }
        }
        if (best_j >= 0 && best < b->opt.alpha_del * mean) {
            delete_image(b, best_j);
            b->last_change = steps_now;
        }
    }
}

void set_control(cfneb_band *b, double ftol, long long move_limit) {
    read_params(b);
    b->h_bp->ftol = ftol;
    b->h_bp->converged = 0;
    b->h_bp->move_limit = move_limit;
    CK(cudaMemcpyAsync(b->dv.bp, b->h_bp, sizeof(BandParams), cudaMemcpyHostToDevice, b->s));
    CK(cudaStreamSynchronize(b->s));
    b->ftol = ftol;
}

// Run up to n_eval steps (each: evaluate, then move unless converged or the
// move budget is spent), pausing for refinement checks.
void run_steps(cfneb_band *b, long long n_eval, bool stop_on_converged, int *status) {
    *status = CFNEB_OK;
    read_params(b);
    long long launched = 0;
    int chunk = 8;
    while (launched < n_eval) {
        long long k = std::min<long long>(n_eval - launched, chunk);
        if (b->opt.adaptive) {
            long long cur = b->h_bp->steps;
            long long to_check = b->opt.k_ref - (cur % b->opt.k_ref);
            k = std::min(k, to_check);
        }
        steps(b, (int)k);
        launched += k;
        read_params(b);
        if (b->h_bp->status) {
            *status = status_from_bits(b->h_bp->status);
            return;
        }
        if (stop_on_converged && b->h_bp->converged) return;
        if (b->opt.adaptive) {
            long long cur = b->h_bp->steps;
            if (cur > 0 && cur % b->opt.k_ref == 0 && cur != b->last_check &&
                cur - b->last_change >= b->opt.cooldown) {
                b->last_check = cur;
                refine(b);
                read_params(b);
            }
        } else {
            chunk = std::min(chunk * 2, 256);
        }
    }
}

cfneb_band *create(const cfneb_structure *A, const cfneb_structure *B, int N,
                   const cfneb_potential *pot, const cfneb_cell_filter *cf,
                   const cfneb_options *opt, void *stream, int *err) {
    *err = CFNEB_OK;
    cfneb_band *b = new cfneb_band();
    b->user = (cudaStream_t)stream;
    b->n = A->n_atoms;
    b->N = N;
    b->opt = *opt;
    if (b->opt.n_max < N) b->opt.n_max = N;
    if (b->opt.n_min < 3) b->opt.n_min = 3;
    b->ncap = b->opt.n_max;
    b->precision = opt->precision;
    b->ts = (opt->precision == CFNEB_MIXED) ? 4 : 8;
    b->kind = pot->kind;
    b->filt = cf ? *cf : cfneb_cell_filter{1, CFNEB_ROTFREE_B, 0.0, 0.0};
    std::memcpy(b->h0, A->cell, sizeof(b->h0));
    b->c = b->filt.cell_factor > 0 ? b->filt.cell_factor : (double)b->n;
    CK(cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
    CK(cudaMallocHost((void **)&b->h_bp, sizeof(BandParams)));
    b->prof_ev.resize(2 * 64);
    for (auto &e : b->prof_ev) CK(cudaEventCreate(&e));

    // potential
    BandParams &P = *b->h_bp;
    std::memset(&P, 0, sizeof(P));
    double rc;
    if (pot->kind == CFNEB_LJ) {
        double eps = pot->eps, sig = pot->sigma;
        rc = pot->rc;
        double sr6 = std::pow(sig / rc, 6.0);
        P.pot[0] = eps;
        P.pot[1] = sig;
        P.pot[2] = rc;
        P.pot[3] = pot->shift_energy ? 4.0 * eps * (sr6 * sr6 - sr6) : 0.0;
    } else {
        bool zero = true;
        for (int k = 0; k < 11; ++k) zero = zero && pot->tersoff[k] == 0.0;
        for (int k = 0; k < 11; ++k) P.pot[k] = zero ? kTersoff1988C[k] : pot->tersoff[k];
        rc = P.pot[9] + P.pot[10];
    }
    double bscale = opt->bin_scale > 0 ? opt->bin_scale : 1.0;
    double bin_w = rc * bscale;
    // geometry
    const int n = b->n, rows = n + 3;
    BandDev &d = b->dv;
    d.n = n;
    d.rows = rows;
    d.ncap = b->ncap;
    int nb0 = bins_for(A->cell, bin_w), nb1 = bins_for(B->cell, bin_w);
    d.nbins_cap = (int)std::min<long long>((long long)(1.5 * std::max(nb0, nb1)) + 64, 1LL << 26);
    d.atpi = (n + TILE - 1) / TILE;
    d.rtpi = (rows + TILE - 1) / TILE;
    const size_t nc = (size_t)b->ncap;
    const size_t vec = nc * rows * 3 * b->ts;
    d.X = dalloc(b, vec);
    d.F = dalloc(b, vec);
    d.Fneb = dalloc(b, vec);
    d.v = dalloc(b, vec);
    d.sc = (ImgScalars *)dalloc(b, nc * sizeof(ImgScalars));
    d.bp = (BandParams *)dalloc(b, sizeof(BandParams));
    d.bin_count = (int *)dalloc(b, nc * d.nbins_cap * sizeof(int));
    d.bin_start = (int *)dalloc(b, nc * (d.nbins_cap + 1) * sizeof(int));
    d.tsum_cap = (d.nbins_cap + 1023) / 1024 + 1;
    d.bin_tsum = (int *)dalloc(b, nc * d.tsum_cap * sizeof(int));
    const size_t na = nc * n;
    d.atom_bin = (int *)dalloc(b, na * sizeof(int));
    d.atom_rank = (int *)dalloc(b, na * sizeof(int));
    d.slot_unsorted = (int *)dalloc(b, na * sizeof(int));
    d.slot_atom = (int *)dalloc(b, na * sizeof(int));
    d.slot_bin = (int *)dalloc(b, na * sizeof(int));
    d.atom_slot = (int *)dalloc(b, na * sizeof(int));
    d.atom_off = dalloc(b, na * 4 * b->ts);
    d.slot_off = dalloc(b, na * 4 * b->ts);
    d.atom_off_lo = dalloc(b, na * 4 * b->ts);
    d.slot_off_lo = dalloc(b, na * 4 * b->ts);
    if (pot->kind == CFNEB_TERSOFF) {
        d.nbr_cnt = (int *)dalloc(b, na * sizeof(int));
        d.nbr_slot = (int *)dalloc(b, na * MAXN_TERSOFF * sizeof(int));
        d.nbr_code = (int *)dalloc(b, na * MAXN_TERSOFF * sizeof(int));
        d.nbr_P = dalloc(b, na * 3 * MAXN_TERSOFF * b->ts);
    }
    d.atom_part = (double *)dalloc(b, nc * d.atpi * NPART * sizeof(double));
    d.row_part = (double *)dalloc(b, nc * d.rtpi * NPART * sizeof(double));
    d.cart = (double *)dalloc(b, na * 3 * sizeof(double));
    b->d_self = (BandDev *)dalloc(b, sizeof(BandDev));
    b->d_atiles = (Tile *)dalloc(b, nc * d.atpi * sizeof(Tile));
    b->d_rtiles = (Tile *)dalloc(b, nc * d.rtpi * sizeof(Tile));
    b->d_imgs = (ImgRef *)dalloc(b, nc * sizeof(ImgRef));
    b->d_band_ids = (int *)dalloc(b, sizeof(int));
    b->d_scratch_tiles =
        (Tile *)dalloc(b, nc * std::max(d.atpi, d.rtpi) * sizeof(Tile));
    b->d_scratch_imgs = (ImgRef *)dalloc(b, nc * sizeof(ImgRef));
    CK(cudaMemsetAsync(d.bin_count, 0, nc * d.nbins_cap * sizeof(int), b->s));
    CK(cudaMemsetAsync(d.v, 0, vec, b->s));
    CK(cudaMemsetAsync(d.Fneb, 0, vec, b->s));
    CK(cudaMemsetAsync(d.F, 0, vec, b->s));
    CK(cudaMemsetAsync(d.sc, 0, nc * sizeof(ImgScalars), b->s));
    int zero = 0;
    CK(cudaMemcpyAsync(b->d_band_ids, &zero, sizeof(int), cudaMemcpyHostToDevice, b->s));
    CK(cudaMemcpyAsync(b->d_self, &d, sizeof(BandDev), cudaMemcpyHostToDevice, b->s));

    // band parameters
    std::memcpy(P.h0, b->h0, sizeof(P.h0));
    inv3(P.h0, P.h0inv);
    P.c = b->c;
    P.pressure = b->filt.pressure;
    P.k = opt->k_spring;
    P.dt0 = opt->dt;
    P.dt_max = opt->dt_max > 0 ? opt->dt_max : 10.0 * opt->dt;
    P.maxstep = opt->maxstep;
    P.rc = rc;
    P.bin_w = bin_w;
    P.ftol = -1.0;
    P.move_limit = 1LL << 62;
    P.filter = b->filt.enabled ? 1 : 0;
    P.variant = b->filt.variant;
    P.climb = opt->climb ? 1 : 0;
    P.n = n;
    P.N = N;
    P.kind = pot->kind;
    P.dt = P.dt0;
    P.alpha = 0.1;
    P.npos = 0;
    P.fresh = 1;
    P.ci = -1;
    CK(cudaMemcpyAsync(d.bp, &P, sizeof(BandParams), cudaMemcpyHostToDevice, b->s));

    // endpoints and interpolation on the device
    double *dR = nullptr;
    size_t rbytes = (size_t)n * 3 * sizeof(double);
    size_t nbytes = opt->interior_noise ? (size_t)(N - 2) * n * 3 * sizeof(double) : 0;
    CK(cudaMalloc(&dR, 2 * rbytes + nbytes + 9 * sizeof(double)));
    double *dR1 = dR + (size_t)n * 3;
    double *dnoise = opt->interior_noise ? dR1 + (size_t)n * 3 : nullptr;
    double *dh1 = dR1 + (size_t)n * 3 + (opt->interior_noise ? (size_t)(N - 2) * n * 3 : 0);
    try {
        CK(cudaMemcpyAsync(dR, A->positions, rbytes, cudaMemcpyHostToDevice, b->s));
        CK(cudaMemcpyAsync(dR1, B->positions, rbytes, cudaMemcpyHostToDevice, b->s));
        if (dnoise)
            CK(cudaMemcpyAsync(dnoise, opt->interior_noise, nbytes, cudaMemcpyHostToDevice, b->s));
        CK(cudaMemcpyAsync(dh1, B->cell, 9 * sizeof(double), cudaMemcpyHostToDevice, b->s));
        if (b->precision == CFNEB_MIXED)
            launch_setup<float>(dR, dR1, dnoise, n, N, b->d_self, b->s, dh1);
        else
            launch_setup<double>(dR, dR1, dnoise, n, N, b->d_self, b->s, dh1);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(b->s));
    } catch (...) {
        cudaFree(dR);
        throw;
    }
    CK(cudaFree(dR));
    build_tables(b);
    eval_images(b, {0, N - 1});
    read_params(b);
    if (b->h_bp->status) *err = status_from_bits(b->h_bp->status);
    return b;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================

extern "C" {

int cfneb_default_options(cfneb_options *o) {
    if (!o) return CFNEB_ERR_INVALID_ARG;
    std::memset(o, 0, sizeof(*o));
    o->k_spring = 0.1;
    o->climb = 1;
    o->precision = CFNEB_FP64;
    o->dt = 0.1;
    o->dt_max = 1.0;
    o->maxstep = 0.2;
    o->interior_noise = nullptr;
    o->adaptive = 0;
    o->n_min = 3;
    o->n_max = 0;
    o->k_ref = 10;
    o->cooldown = 20;
    o->alpha_ins = 1.5;
    o->alpha_del = 0.5;
    o->bin_scale = 0.0;
    return CFNEB_OK;
}

int cfneb_create_band(const cfneb_structure *initial, const cfneb_structure *final_,
                      int32_t n_images, const cfneb_potential *potential,
                      const cfneb_cell_filter *cell_filter, const cfneb_options *options,
                      void *cuda_stream, cfneb_band **out) {
    if (!initial || !final_ || !potential || !out || n_images < 3) return CFNEB_ERR_INVALID_ARG;
    *out = nullptr;
    if (!initial->positions || !final_->positions || initial->n_atoms <= 0)
        return CFNEB_ERR_INVALID_ARG;
    if (initial->n_atoms != final_->n_atoms) return CFNEB_ERR_SHAPE_MISMATCH;
    if (initial->types && final_->types) {
        for (int i = 0; i < initial->n_atoms; ++i)
            if (initial->types[i] != final_->types[i]) return CFNEB_ERR_SHAPE_MISMATCH;
    }
    if (initial->types)
        for (int i = 1; i < initial->n_atoms; ++i)
            if (initial->types[i] != initial->types[0]) return CFNEB_ERR_INVALID_ARG;
    if (potential->kind != CFNEB_LJ && potential->kind != CFNEB_TERSOFF)
        return CFNEB_ERR_INVALID_ARG;
    if (potential->kind == CFNEB_LJ &&
        (potential->rc <= 0 || potential->sigma <= 0 || potential->eps <= 0))
        return CFNEB_ERR_INVALID_ARG;
    if (std::fabs(det3(initial->cell)) <= 0 || std::fabs(det3(final_->cell)) <= 0)
        return CFNEB_ERR_INVALID_ARG;
    cfneb_options opt;
    if (options) opt = *options;
    else cfneb_default_options(&opt);
    if (opt.precision != CFNEB_FP64 && opt.precision != CFNEB_MIXED) return CFNEB_ERR_INVALID_ARG;
    if (opt.dt <= 0 || opt.maxstep <= 0) return CFNEB_ERR_INVALID_ARG;
    if (opt.k_ref <= 0) opt.k_ref = 10;
    if (opt.bin_scale != 0 && opt.bin_scale < 0.25) return CFNEB_ERR_INVALID_ARG;
    if (cell_filter && cell_filter->variant != CFNEB_ROTFREE_B &&
        cell_filter->variant != CFNEB_DEFGRAD_D)
        return CFNEB_ERR_INVALID_ARG;
    cfneb_band *b = nullptr;
    int err = CFNEB_OK;
    try {
        b = create(initial, final_, n_images, potential, cell_filter, &opt, cuda_stream, &err);
        leave(b);
    } catch (CudaFail &f) {
        free_band(b);
        return f.e == cudaErrorMemoryAllocation ? CFNEB_ERR_OUT_OF_MEMORY : CFNEB_ERR_CUDA;
    }
    if (err != CFNEB_OK) {
        free_band(b);
        return err;
    }
    *out = b;
    return CFNEB_OK;
}

int cfneb_step(cfneb_band *b, int32_t n_steps) {
    if (!b || n_steps < 0) return CFNEB_ERR_INVALID_ARG;
    try {
        enter(b);
        int st = CFNEB_OK;
        if (b->opt.adaptive) run_steps(b, n_steps, false, &st);
        else steps(b, n_steps);
        leave(b);
        return st;
    } catch (CudaFail &) {
        return CFNEB_ERR_CUDA;
    }
}

int cfneb_relax(cfneb_band *b, double fmax, int64_t max_steps, int64_t *steps_done,
                int32_t *converged) {
    if (!b || max_steps < 0 || !(fmax >= 0)) return CFNEB_ERR_INVALID_ARG;
    try {
        enter(b);
        read_params(b);
        const long long start = b->h_bp->steps;
        // at most max_steps moves, max_steps + 1 evaluations: the test comes
        // before each move, and once more after the last one
        set_control(b, fmax, start + max_steps);
        int st = CFNEB_OK;
        run_steps(b, max_steps + 1, true, &st);
        read_params(b);
        const long long done = b->h_bp->steps - start;
        const int conv = b->h_bp->converged ? 1 : 0;
        set_control(b, fmax, 1LL << 62);
        leave(b);
        if (steps_done) *steps_done = done;
        if (converged) *converged = conv;
        if (st != CFNEB_OK) return st;
        return conv ? CFNEB_OK : CFNEB_NOT_CONVERGED;
    } catch (CudaFail &) {
        return CFNEB_ERR_CUDA;
    }
}

int cfneb_insert_image(cfneb_band *b, int32_t after_index) {
    if (!b) return CFNEB_ERR_INVALID_ARG;
    try {
        enter(b);
        int st = insert_image(b, after_index);
        leave(b);
        return st;
    } catch (CudaFail &) {
        return CFNEB_ERR_CUDA;
    }
}

int cfneb_delete_image(cfneb_band *b, int32_t index) {
    if (!b) return CFNEB_ERR_INVALID_ARG;
    try {
        enter(b);
        int st = delete_image(b, index);
        leave(b);
        return st;
    } catch (CudaFail &) {
        return CFNEB_ERR_CUDA;
    }
}

int cfneb_get_path(const cfneb_band *cb, int32_t *n_images, double *positions, double *cells,
                   double *energies, double *fmax) {
    cfneb_band *b = const_cast<cfneb_band *>(cb);
    if (!b) return CFNEB_ERR_INVALID_ARG;
    try {
        enter(b);
        if (n_images) *n_images = b->N;
        if (positions || cells || energies) {
            // FP64 energies of the current images (map-back, cell list, energy),
            // then Cartesian positions R = R~ D from the same map-back
            refine_energies(b, 0, b->N);
            if (b->precision == CFNEB_MIXED)
                launch_cartesian<float>(b->d_scratch_imgs, b->N, b->n, b->d_self, b->s);
            else
                launch_cartesian<double>(b->d_scratch_imgs, b->N, b->n, b->d_self, b->s);
            CK(cudaGetLastError());
        }
        std::vector<ImgScalars> sc(b->N);
        CK(cudaMemcpyAsync(sc.data(), b->dv.sc, b->N * sizeof(ImgScalars),
                           cudaMemcpyDeviceToHost, b->s));
        if (positions)
            CK(cudaMemcpyAsync(positions, b->dv.cart, (size_t)b->N * b->n * 3 * sizeof(double),
                               cudaMemcpyDeviceToHost, b->s));
        read_params(b);
        for (int i = 0; i < b->N; ++i) {
            if (cells) std::memcpy(cells + 9 * i, sc[i].h, 9 * sizeof(double));
            if (energies) energies[i] = sc[i].E64;
        }
        if (fmax) *fmax = b->h_bp->fmax;
        leave(b);
        return status_from_bits(b->h_bp->status);
    } catch (CudaFail &) {
        return CFNEB_ERR_CUDA;
    }
}

int cfneb_get_state(const cfneb_band *cb, double *X, double *F, double *Fneb, double *virials,
                    double *fire, int32_t *climbing_index) {
    cfneb_band *b = const_cast<cfneb_band *>(cb);
    if (!b) return CFNEB_ERR_INVALID_ARG;
    try {
        enter(b);
        const size_t cnt = (size_t)b->N * b->dv.rows * 3;
        std::vector<char> tmp(cnt * b->ts);
        auto fetch = [&](void *src, double *dst) {
            if (!dst) return;
            CK(cudaMemcpyAsync(tmp.data(), src, cnt * b->ts, cudaMemcpyDeviceToHost, b->s));
            CK(cudaStreamSynchronize(b->s));
            if (b->ts == 4) {
                const float *f = (const float *)tmp.data();
                for (size_t i = 0; i < cnt; ++i) dst[i] = f[i];
            } else {
                std::memcpy(dst, tmp.data(), cnt * sizeof(double));
            }
        };
        fetch(b->dv.X, X);
        fetch(b->dv.F, F);
        fetch(b->dv.Fneb, Fneb);
        if (Fneb) {  // endpoints carry no NEB force
            std::memset(Fneb, 0, (size_t)b->dv.rows * 3 * sizeof(double));
            std::memset(Fneb + (size_t)(b->N - 1) * b->dv.rows * 3, 0,
                        (size_t)b->dv.rows * 3 * sizeof(double));
        }
        std::vector<ImgScalars> sc(b->N);
        CK(cudaMemcpyAsync(sc.data(), b->dv.sc, b->N * sizeof(ImgScalars),
                           cudaMemcpyDeviceToHost, b->s));
        read_params(b);
        if (virials)
            for (int i = 0; i < b->N; ++i) std::memcpy(virials + 9 * i, sc[i].V, 9 * sizeof(double));
        if (fire) {
            fire[0] = b->h_bp->dt;
            fire[1] = b->h_bp->alpha;
            fire[2] = b->h_bp->npos;
            fire[3] = (double)b->h_bp->steps;
        }
        if (climbing_index) *climbing_index = b->h_bp->ci;
        leave(b);
        return status_from_bits(b->h_bp->status);
    } catch (CudaFail &) {
        return CFNEB_ERR_CUDA;
    }
}

int cfneb_destroy_band(cfneb_band *b) {
    if (!b) return CFNEB_ERR_INVALID_ARG;
    try {
        enter(b);
    } catch (CudaFail &) {
    }
    free_band(b);
    return CFNEB_OK;
}

int cfneb_evaluate(const cfneb_structure *structures, int32_t count,
                   const cfneb_potential *potential, int32_t precision, void *cuda_stream,
                   double *energies, double *forces, double *virials) {
    if (!structures || count <= 0 || !potential) return CFNEB_ERR_INVALID_ARG;
    size_t off = 0;
    for (int k = 0; k < count; ++k) {
        const cfneb_structure &S = structures[k];
        // each structure is the middle image of a three-image band whose
        // reference cell is its own cell (D = I, forces are Cartesian)
        cfneb_options opt;
        cfneb_default_options(&opt);
        opt.precision = precision;
        cfneb_cell_filter cf{1, CFNEB_ROTFREE_B, 0.0, 0.0};
        cfneb_band *b = nullptr;
        int st = cfneb_create_band(&S, &S, 3, potential, &cf, &opt, cuda_stream, &b);
        if (st != CFNEB_OK) return st;
        try {
            enter(b);
            // the endpoints were evaluated at creation: image 0 is S; its
            // reported energy is the FP64 one
            refine_energies(b, 0, 1);
            std::vector<ImgScalars> sc(1);
            CK(cudaMemcpyAsync(sc.data(), b->dv.sc, sizeof(ImgScalars), cudaMemcpyDeviceToHost,
                               b->s));
            std::vector<char> tmp((size_t)b->dv.rows * 3 * b->ts);
            CK(cudaMemcpyAsync(tmp.data(), b->dv.F, tmp.size(), cudaMemcpyDeviceToHost, b->s));
            CK(cudaStreamSynchronize(b->s));
            if (energies) energies[k] = sc[0].E64;
            if (virials) std::memcpy(virials + 9 * k, sc[0].V, 9 * sizeof(double));
            if (forces) {
                for (int i = 0; i < S.n_atoms * 3; ++i)
                    forces[off + i] = b->ts == 4 ? ((const float *)tmp.data())[i]
                                                 : ((const double *)tmp.data())[i];
            }
            leave(b);
        } catch (CudaFail &) {
            cfneb_destroy_band(b);
            return CFNEB_ERR_CUDA;
        }
        off += (size_t)S.n_atoms * 3;
        cfneb_destroy_band(b);
    }
    return CFNEB_OK;
}

int cfneb_profile(cfneb_band *b, int32_t enable) {
    if (!b) return CFNEB_ERR_INVALID_ARG;
    b->prof = enable != 0;
    for (int k = 0; k < K_COUNT; ++k) {
        b->prof_ms[k] = 0.0;
        b->prof_n[k] = 0;
    }
    return CFNEB_OK;
}

int cfneb_profile_read(cfneb_band *b, int32_t kernel_id, double *total_ms, int64_t *launches) {
    if (!b || kernel_id < 0 || kernel_id >= K_COUNT) return CFNEB_ERR_INVALID_ARG;
    if (total_ms) *total_ms = b->prof_ms[kernel_id];
    if (launches) *launches = b->prof_n[kernel_id];
    return CFNEB_OK;
}

int32_t cfneb_kernel_count(void) { return K_COUNT; }

const char *cfneb_kernel_name(int32_t id) {
    return (id >= 0 && id < K_COUNT) ? kKernelNames[id] : "unknown";
}

int cfneb_get_work(const cfneb_band *cb, double *pairs, double *triples) {
    cfneb_band *b = const_cast<cfneb_band *>(cb);
    if (!b) return CFNEB_ERR_INVALID_ARG;
    try {
        enter(b);
        std::vector<ImgScalars> sc(b->N);
        CK(cudaMemcpyAsync(sc.data(), b->dv.sc, b->N * sizeof(ImgScalars),
                           cudaMemcpyDeviceToHost, b->s));
        CK(cudaStreamSynchronize(b->s));
        double p = 0.0, t = 0.0;
        for (int i = 1; i < b->N - 1; ++i) {
            p += sc[i].pairs;
            t += sc[i].triples;
        }
        if (pairs) *pairs = p;
        if (triples) *triples = t;
        leave(b);
        return CFNEB_OK;
    } catch (CudaFail &) {
        return CFNEB_ERR_CUDA;
    }
}

int cfneb_launches_per_step(const cfneb_band *b, int32_t *launches) {
    if (!b || !launches) return CFNEB_ERR_INVALID_ARG;
    *launches = launches_per_step(b);
    return CFNEB_OK;
}

const char *cfneb_status_string(int s) {
    switch (s) {
    case CFNEB_OK: return "ok";
    case CFNEB_NOT_CONVERGED: return "not converged";
    case CFNEB_ERR_INVALID_ARG: return "invalid argument";
    case CFNEB_ERR_SHAPE_MISMATCH: return "endpoint shape mismatch";
    case CFNEB_ERR_OUT_OF_MEMORY: return "device out of memory";
    case CFNEB_ERR_HBM_BUDGET: return "memory budget exceeded";
    case CFNEB_ERR_CUDA: return g_last_error.empty() ? "CUDA error" : g_last_error.c_str();
    case CFNEB_ERR_NONFINITE: return "non-finite value";
    case CFNEB_ERR_NOT_SPD: return "lattice coordinate not positive definite";
    case CFNEB_ERR_NBR_OVERFLOW: return "neighbour capacity exceeded";
    case CFNEB_ERR_TIMEOUT: return "device wait timed out";
    case CFNEB_ERR_STATE: return "invalid state for this call";
    default: return "unknown status";
    }
}

}  // extern "C"
