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
#include <chrono>
#include <cmath>
#include <deque>
#include <thread>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
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

static_assert(NEP_NW == CFNEB_NEP_N_WEIGHTS, "NEP weight count of the header and kernels");
static_assert(KIND_LJ == CFNEB_LJ && KIND_TERSOFF == CFNEB_TERSOFF && KIND_NEP == CFNEB_NEP,
              "potential kinds of the header and kernels");

enum KernelId {
    K_MAPBACK, K_BIN_ASSIGN, K_BIN_TILESUM, K_BIN_TILESCAN, K_BIN_SCANFILL, K_BIN_SCATTER,
    K_BIN_ORDER, K_LJ, K_TERS_LIST, K_TERS_REVERSE, K_TERS_PARTIALS, K_TERS_GATHER, K_IMAGE_FINALIZE,
    K_BAND_DOTS, K_DOTS_REDUCE, K_NEB_COEF, K_NEB_FORCE, K_FIRE_SCALARS, K_FIRE_UPDATE, K_LJ_LIST,
    K_LJ_CELLS, K_NEP_PARTIALS, K_COUNT
};
const char *kKernelNames[K_COUNT] = {
    "mapback", "bin_assign", "bin_tilesum", "bin_tilescan", "bin_scanfill", "bin_scatter",
    "bin_order", "lj_force", "tersoff_list", "tersoff_reverse", "tersoff_partials", "tersoff_gather",
    "image_finalize", "band_dots", "dots_reduce", "neb_coef", "neb_force", "fire_scalars",
    "fire_update", "lj_list", "lj_force_cells", "nep_partials"};

const double kTersoff1988C[11] = {1393.6, 346.74, 3.4879, 2.2119, 1.5724e-7, 0.72751,
                                  38049.0, 4.3484, -0.57058, 1.95, 0.15};

// bin width candidates (x cutoff) of the autotuner; the first is the finest
const double kTuneScales[4] = {0.5, 0.75, 1.0, 1.3};
// resident blocks per SM of the FP32 force kernels (the register cap of the
// kernel variant launched): defaults and the autotuner's candidates
constexpr int kLjMinb = 7, kTersMinb = 5;
const int kLjMinbs[4] = {5, 6, 7, 8};
const int kTersMinbs[5] = {4, 5, 6, 7, 8};

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, double> g_tune;  // class -> bin width / rc
std::map<std::tuple<int, int, int, int>, int> g_tune_minb;  // class -> blocks per SM

// untuned default per potential (measured on GB300: LJ at FCC density is
// fastest with half-cutoff bins, carbon Tersoff with cutoff-wide bins)
int tuned_minb(const std::tuple<int, int, int, int> &key) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_minb.find(key);
    if (it != g_tune_minb.end()) return it->second;
    return 0;  // the kernel's default
}

double tuned_scale(const std::tuple<int, int, int, int> &key) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second;
    return std::get<0>(key) == CFNEB_LJ ? 0.5 : 1.0;
}

}  // namespace

struct cfneb_batch;
namespace {
void batch_mark_dirty(cfneb_batch *bt);
}

// One band: its device buffers and host-side configuration.
// A side stream and two events: inside a graph capture, work recorded on
// the side stream after `a` runs beside the main stream until the main
// stream waits on `b` (a fork and a join in the captured graph).
struct Fork {
    cudaStream_t s = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    void create() {
        CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&a, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&b, cudaEventDisableTiming));
    }
    void destroy() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
        if (s) cudaStreamDestroy(s);
        s = nullptr;
        a = b = nullptr;
    }
};

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
    long long move_limit = 1LL << 62;  // host copy of BandParams::move_limit
    double rc = 0.0;             // potential cutoff
    double rl = 0.0;             // list cutoff rc + skin
    std::tuple<int, int, int, int> tune_key{};
    int minb = 0;                // force kernel blocks per SM (0: the default)
    double ftol = -1.0;
    bool ends_e64 = false;       // the endpoints' FP64 energies are known
    // stream ordering
    cudaStream_t user = nullptr, s = nullptr;
    cudaStream_t s_body = nullptr;   // captures the conditional list-rebuild body
    Fork fork;                       // the finalize beside the force gather (graphs)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // launch tables (device) and their sizes
    Tile *d_atiles = nullptr;    // atom tiles of the interior images
    Tile *d_rtiles = nullptr;    // row tiles of the interior images
    ImgRef *d_imgs = nullptr;    // interior images
    int *d_band_ids = nullptr;
    Tile *d_scratch_tiles = nullptr;   // tables for ad-hoc image sets
    ImgRef *d_scratch_imgs = nullptr;
    int n_atiles = 0, n_rtiles = 0, n_imgs = 0;
    // graphs: one step, and GRAPH_STEPS steps
    cudaGraphExec_t gexec = nullptr, gexec_n = nullptr;
    bool graph_dirty = true;
    // profiling
    bool prof = false;
    double prof_ms[K_COUNT]{};
    long long prof_n[K_COUNT]{};
    std::vector<cudaEvent_t> prof_ev;
    // pinned host mirror of BandParams
    BandParams *h_bp = nullptr;
    // batch membership: while a member, s is the batch's stream
    cfneb_batch *batch = nullptr;
    cudaStream_t own_s = nullptr;
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
    if (b->own_s) b->s = b->own_s;
    for (void *p : b->allocs) cudaFree(p);
    b->allocs.clear();
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->gexec_n) cudaGraphExecDestroy(b->gexec_n);
    for (auto e : b->prof_ev) cudaEventDestroy(e);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->s) cudaStreamDestroy(b->s);
    if (b->s_body) cudaStreamDestroy(b->s_body);
    b->fork.destroy();
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

// every perpendicular width of h is at least rl / MAX_STENCIL (with a
// margin for the FP32 bin arithmetic)
bool stencil_reaches(const double *h, double rl) {
    double w[3];
    widths(h, w);
    for (int a = 0; a < 3; ++a)
        if (!(rl < MAX_STENCIL * w[a] * 0.999)) return false;
    return true;
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
    if (b->batch) batch_mark_dirty(b->batch);
}

// ---- kernel sequences ------------------------------------------------------

// Kernel launches of one step (or one evaluation) over a set of images, possibly
// of many bands: the tables index into an array of BandDev.
struct LaunchSet {
    BandDev *d_bands = nullptr;
    cudaStream_t s = nullptr;
    const ImgRef *imgs = nullptr;
    int nimg = 0;
    const Tile *atiles = nullptr;        // atom tiles of every listed image
    int n_atiles = 0;
    const Tile *atiles_lj = nullptr;     // atom tiles of the LJ bands with a neighbour list
    int n_lj = 0;
    const Tile *atiles_ljc = nullptr;    // atom tiles of the LJ bands without one
    int n_ljc = 0;
    const Tile *atiles_ters = nullptr;   // the Tersoff bands' atom tiles
    int n_ters = 0;
    const Tile *atiles_nep = nullptr;    // the NEP bands' atom tiles
    int n_nep = 0;
    const Tile *rtiles = nullptr;        // row tiles
    int n_rtiles = 0;
    const int *band_ids = nullptr;
    int nbands = 0;
    int max_bins = 0;                    // largest nbins_cap among the bands
    int force_rebuild = 0;               // rebuild every listed image's cell list
    int lj_minb = kLjMinb, ters_minb = kTersMinb;  // force kernel variants
    cudaStream_t s_body = nullptr;       // captures the conditional rebuild body
    const Fork *fork = nullptr;          // side stream and events for the finalize
};

// optional CUDA-event bracketing of every launch (profiling)
struct Launcher {
    bool prof = false;
    std::vector<cudaEvent_t> *ev = nullptr;
    cudaStream_t s = nullptr;
    int k = 0;
    std::vector<int> ids;
    void pre(int) {
        if (prof) CK(cudaEventRecord((*ev)[2 * k], s));
    }
    void post(int id) {
        if (prof) {
            CK(cudaEventRecord((*ev)[2 * k + 1], s));
            ids.push_back(id);
            ++k;
        }
    }
};

// cell-list scan, scatter and order, then the neighbour lists (they index
// cell-list slots, so they are rebuilt with every cell list, also by an
// energy-only evaluation); each kernel skips the images that keep theirs
template <typename T>
void enqueue_rebuild(const LaunchSet &ls, Launcher &L) {
    BandDev *d = ls.d_bands;
    cudaStream_t s = ls.s;
    L.pre(K_BIN_TILESUM); launch_bin_scan(ls.imgs, ls.nimg, ls.max_bins, d, s, 0); L.post(K_BIN_TILESUM);
    L.pre(K_BIN_TILESCAN); launch_bin_scan(ls.imgs, ls.nimg, ls.max_bins, d, s, 1); L.post(K_BIN_TILESCAN);
    L.pre(K_BIN_SCANFILL); launch_bin_scan(ls.imgs, ls.nimg, ls.max_bins, d, s, 2); L.post(K_BIN_SCANFILL);
    L.pre(K_BIN_SCATTER); launch_bin_scatter(ls.atiles, ls.n_atiles, d, s); L.post(K_BIN_SCATTER);
    L.pre(K_BIN_ORDER); launch_bin_order<T>(ls.imgs, ls.nimg, ls.max_bins, d, s); L.post(K_BIN_ORDER);
    // the neighbour lists index cell-list slots: they are rebuilt with every
    // cell list, also by an energy-only evaluation
    if (ls.n_lj) {
        L.pre(K_LJ_LIST); launch_lj_list<T>(ls.atiles_lj, ls.n_lj, d, s); L.post(K_LJ_LIST);
    }
    if (ls.n_ters) {
        L.pre(K_TERS_LIST); launch_tersoff_list<T>(ls.atiles_ters, ls.n_ters, d, s);
        L.post(K_TERS_LIST);
        L.pre(K_TERS_REVERSE); launch_tersoff_reverse<T>(ls.atiles_ters, ls.n_ters, d, s);
        L.post(K_TERS_REVERSE);
    }
    // NEP bands use the same many-body lists
    if (ls.n_nep) {
        L.pre(K_TERS_LIST); launch_tersoff_list<T>(ls.atiles_nep, ls.n_nep, d, s);
        L.post(K_TERS_LIST);
        L.pre(K_TERS_REVERSE); launch_tersoff_reverse<T>(ls.atiles_nep, ls.n_nep, d, s);
        L.post(K_TERS_REVERSE);
    }
}

template <typename T>
void enqueue_eval_set(const LaunchSet &ls, Launcher &L, bool forces = true) {
    BandDev *d = ls.d_bands;
    cudaStream_t s = ls.s;
    // the displacements since the last build were taken by the last move
    // (k_fire_update); then map-back and the list decision
    L.pre(K_MAPBACK); launch_mapback<T>(ls.imgs, ls.nimg, d, ls.force_rebuild, s);
    L.post(K_MAPBACK);
    // the cell-list and neighbour-list rebuild: inside a graph capture it
    // goes into the body of a conditional node that runs only in steps
    // where some image rebuilds (most steps keep every list; bin_assign
    // switches the node on); outside a capture its kernels run and skip the
    // images that keep their lists
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(s, &cst));
    const bool cond_node = cst == cudaStreamCaptureStatusActive && ls.s_body && !L.prof;
    cudaGraphConditionalHandle cond = 0;
    if (cond_node) {
        cudaGraph_t graph = nullptr;
        CK(cudaStreamGetCaptureInfo(s, &cst, nullptr, &graph, nullptr, nullptr, nullptr));
        CK(cudaGraphConditionalHandleCreate(&cond, graph, 0, cudaGraphCondAssignDefault));
    }
    L.pre(K_BIN_ASSIGN);
    launch_bin_assign<T>(ls.atiles, ls.n_atiles, d, s, cond, cond_node ? 1 : 0);
    L.post(K_BIN_ASSIGN);
    if (cond_node) {
        cudaGraph_t graph = nullptr;
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        CK(cudaStreamGetCaptureInfo(s, &cst, nullptr, &graph, &deps, nullptr, &nd));
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = cond;
        cp.conditional.type = cudaGraphCondTypeIf;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        CK(cudaGraphAddNode(&node, graph, deps, nullptr, nd, &cp));
        CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1,
                                               cudaStreamSetCaptureDependencies));
        CK(cudaStreamBeginCaptureToGraph(ls.s_body, cp.conditional.phGraph_out[0], nullptr,
                                         nullptr, 0, cudaStreamCaptureModeThreadLocal));
        LaunchSet body = ls;
        body.s = ls.s_body;
        try {
            enqueue_rebuild<T>(body, L);
        } catch (...) {
            cudaGraph_t tmp = nullptr;
            cudaStreamEndCapture(ls.s_body, &tmp);
            throw;
        }
        cudaGraph_t tmp = nullptr;
        CK(cudaStreamEndCapture(ls.s_body, &tmp));
    } else {
        enqueue_rebuild<T>(ls, L);
    }
    if (!forces) {
        launch_energy64<T>(ls.atiles, ls.n_atiles, ls.imgs, ls.nimg, d, s);
        return;
    }
    if (ls.n_lj) {
        L.pre(K_LJ); launch_lj_nbr<T>(ls.atiles_lj, ls.n_lj, d, s, ls.lj_minb); L.post(K_LJ);
    }
    if (ls.n_ljc) {
        L.pre(K_LJ_CELLS); launch_lj<T>(ls.atiles_ljc, ls.n_ljc, d, s); L.post(K_LJ_CELLS);
    }
    if (ls.n_ters) {
        L.pre(K_TERS_PARTIALS);
        launch_tersoff_partials<T>(ls.atiles_ters, ls.n_ters, d, s, ls.ters_minb);
        L.post(K_TERS_PARTIALS);
    }
    if (ls.n_nep) {
        L.pre(K_NEP_PARTIALS); launch_nep_partials<T>(ls.atiles_nep, ls.n_nep, d, s);
        L.post(K_NEP_PARTIALS);
    }
    // Inside a graph the finalize (tile sums into E and V, the lattice
    // force) needs only the partials' records, not the gathered atom
    // forces: it runs on the side stream beside the gathers, joined before
    // the band passes.
    CK(cudaStreamIsCapturing(s, &cst));
    const bool fork = ls.fork && (ls.n_ters || ls.n_nep) && !L.prof &&
                      cst == cudaStreamCaptureStatusActive;
    if (fork) {
        CK(cudaEventRecord(ls.fork->a, s));
        CK(cudaStreamWaitEvent(ls.fork->s, ls.fork->a, 0));
        launch_image_finalize<T>(ls.imgs, ls.nimg, d, ls.fork->s);
        CK(cudaEventRecord(ls.fork->b, ls.fork->s));
    }
    if (ls.n_ters) {
        L.pre(K_TERS_GATHER); launch_tersoff_gather<T>(ls.atiles_ters, ls.n_ters, d, s);
        L.post(K_TERS_GATHER);
    }
    if (ls.n_nep) {
        L.pre(K_TERS_GATHER); launch_tersoff_gather<T>(ls.atiles_nep, ls.n_nep, d, s);
        L.post(K_TERS_GATHER);
    }
    if (fork) {
        CK(cudaStreamWaitEvent(s, ls.fork->b, 0));
    } else {
        L.pre(K_IMAGE_FINALIZE); launch_image_finalize<T>(ls.imgs, ls.nimg, d, s);
        L.post(K_IMAGE_FINALIZE);
    }
}

template <typename T>
void enqueue_step_set(const LaunchSet &ls, Launcher &L) {
    BandDev *d = ls.d_bands;
    cudaStream_t s = ls.s;
    enqueue_eval_set<T>(ls, L);
    L.pre(K_BAND_DOTS); launch_band_dots<T>(ls.rtiles, ls.n_rtiles, d, s); L.post(K_BAND_DOTS);
    L.pre(K_NEB_FORCE); launch_neb_force<T>(ls.rtiles, ls.n_rtiles, d, s); L.post(K_NEB_FORCE);
    L.pre(K_FIRE_UPDATE); launch_fire_update<T>(ls.rtiles, ls.n_rtiles, ls.imgs, ls.nimg, d, s);
    L.post(K_FIRE_UPDATE);
}

// launches of a step when it rebuilds lists (the graph's conditional node
// skips the 5 cell-list and 1-2 neighbour-list kernels in other steps):
// map-back, bin_assign and the 5 list kernels, the force kernels, the
// finalize and the three band passes
int launches_in_set(const LaunchSet &ls) {
    return 7 + (ls.n_lj ? 2 : 0) + (ls.n_ljc ? 1 : 0) + (ls.n_ters ? 4 : 0) + (ls.n_nep ? 4 : 0) +
           1 + 3;
}

LaunchSet band_set(cfneb_band *b, const ImgRef *imgs, int nimg, const Tile *atiles, int nat) {
    LaunchSet ls;
    ls.d_bands = b->d_self;
    ls.s = b->s;
    ls.imgs = imgs;
    ls.nimg = nimg;
    ls.atiles = atiles;
    ls.n_atiles = nat;
    if (b->kind == CFNEB_LJ && b->dv.lj_cap > 0) {
        ls.atiles_lj = atiles;
        ls.n_lj = nat;
    } else if (b->kind == CFNEB_LJ) {
        ls.atiles_ljc = atiles;
        ls.n_ljc = nat;
    } else if (b->kind == CFNEB_NEP) {
        ls.atiles_nep = atiles;
        ls.n_nep = nat;
    } else {
        ls.atiles_ters = atiles;
        ls.n_ters = nat;
    }
    ls.rtiles = b->d_rtiles;
    ls.n_rtiles = b->n_rtiles;
    ls.band_ids = b->d_band_ids;
    ls.nbands = 1;
    ls.max_bins = b->dv.nbins_cap;
    ls.s_body = b->s_body;
    ls.fork = &b->fork;
    if (b->minb > 0) {
        if (b->kind == CFNEB_LJ) ls.lj_minb = b->minb;
        if (b->kind == CFNEB_TERSOFF) ls.ters_minb = b->minb;
    }
    return ls;
}

LaunchSet band_step_set(cfneb_band *b) {
    return band_set(b, b->d_imgs, b->n_imgs, b->d_atiles, b->n_atiles);
}

template <typename T>
void enqueue_eval(cfneb_band *b, Launcher &L, const ImgRef *imgs, int nimg, const Tile *atiles,
                  int natiles, bool forces = true) {
    // ad-hoc image sets (endpoints, new images, reported energies) are
    // evaluated from freshly built cell lists
    LaunchSet ls = band_set(b, imgs, nimg, atiles, natiles);
    ls.force_rebuild = 1;
    enqueue_eval_set<T>(ls, L, forces);
}

int launches_per_step(const cfneb_band *b) {
    return launches_in_set(band_set(const_cast<cfneb_band *>(b), nullptr, 1, nullptr, 1));
}

// run the launches of `ls` once with events around each launch and add the
// times to (ms, n)
template <typename F>
void profiled(cudaStream_t s, std::vector<cudaEvent_t> &ev, double *ms, long long *n, F enq) {
    Launcher L;
    L.prof = true;
    L.ev = &ev;
    L.s = s;
    enq(L);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    for (int q = 0; q < L.k; ++q) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, ev[2 * q], ev[2 * q + 1]));
        ms[L.ids[q]] += t;
        n[L.ids[q]] += 1;
    }
}

// capture the launches of `enq` on stream s into an executable graph
template <typename F>
cudaGraphExec_t capture(cudaStream_t s, F enq) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    Launcher L;
    try {
        enq(L);
    } catch (...) {
        cudaStreamEndCapture(s, &g);
        if (g) cudaGraphDestroy(g);
        throw;
    }
    CK(cudaStreamEndCapture(s, &g));
    cudaGraphExec_t ge = nullptr;
    cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    CK(e);
    return ge;
}

// Steps per multi-step graph: n steps run as n / GRAPH_STEPS launches of a
// graph of GRAPH_STEPS captured steps and n % GRAPH_STEPS of the one-step
// graph, so that the gap between two graph launches is paid once per
// GRAPH_STEPS steps.  Every step of a graph is the same captured sequence
// (the kernels read the band's state from device memory).
constexpr int GRAPH_STEPS = 8;

void drop_graphs(cudaGraphExec_t &one, cudaGraphExec_t &many) {
    if (one) CK(cudaGraphExecDestroy(one));
    if (many) CK(cudaGraphExecDestroy(many));
    one = many = nullptr;
}

template <typename F>
void launch_steps(cudaGraphExec_t &one, cudaGraphExec_t &many, cudaStream_t s, int n, F enq) {
    if (n >= GRAPH_STEPS && !many)
        many = capture(s, [&](Launcher &L) {
            for (int k = 0; k < GRAPH_STEPS; ++k) enq(L);
        });
    if (n % GRAPH_STEPS && !one) one = capture(s, enq);
    for (int i = 0; i < n / GRAPH_STEPS; ++i) CK(cudaGraphLaunch(many, s));
    for (int i = 0; i < n % GRAPH_STEPS; ++i) CK(cudaGraphLaunch(one, s));
}

void steps(cfneb_band *b, int n) {
    if (n <= 0 || b->N < 3) return;
    const LaunchSet ls = band_step_set(b);
    auto enq = [&](Launcher &L) {
        if (b->precision == CFNEB_MIXED) enqueue_step_set<float>(ls, L);
        else enqueue_step_set<double>(ls, L);
    };
    if (b->prof) {
        for (int i = 0; i < n; ++i) profiled(b->s, b->prof_ev, b->prof_ms, b->prof_n, enq);
        return;
    }
    if (b->graph_dirty) {
        drop_graphs(b->gexec, b->gexec_n);
        b->graph_dirty = false;
    }
    launch_steps(b->gexec, b->gexec_n, b->s, n, enq);
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
    Launcher L;
    if (b->precision == CFNEB_MIXED)
        enqueue_eval<float>(b, L, b->d_scratch_imgs, (int)im.size(), b->d_scratch_tiles,
                            (int)at.size());
    else
        enqueue_eval<double>(b, L, b->d_scratch_imgs, (int)im.size(), b->d_scratch_tiles,
                             (int)at.size());
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(b->s));
}

// FP64 energies (ImgScalars::E64) of the images' current coordinates:
// map-back, cell list and the FP64 energy kernel, no forces
void refine_energies(cfneb_band *b, const std::vector<int> &imgs) {
    std::vector<ImgRef> im;
    std::vector<Tile> at;
    for (int i : imgs) {
        im.push_back({0, i});
        for (int t = 0; t < b->dv.atpi; ++t) at.push_back({0, i, t, 0});
    }
    if (im.empty()) return;
    CK(cudaMemcpyAsync(b->d_scratch_imgs, im.data(), im.size() * sizeof(ImgRef),
                       cudaMemcpyHostToDevice, b->s));
    CK(cudaMemcpyAsync(b->d_scratch_tiles, at.data(), at.size() * sizeof(Tile),
                       cudaMemcpyHostToDevice, b->s));
    Launcher L;
    if (b->precision == CFNEB_MIXED)
        enqueue_eval<float>(b, L, b->d_scratch_imgs, (int)im.size(), b->d_scratch_tiles,
                            (int)at.size(), false);
    else
        enqueue_eval<double>(b, L, b->d_scratch_imgs, (int)im.size(), b->d_scratch_tiles,
                             (int)at.size(), false);
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

// The lattice rows of X are stored as c (B - I) (c (D - I) for the
// deformation-gradient filter); the C ABI exchanges X = (R~, c B).  sign +1
// turns stored rows into the ABI's, -1 the other way (one image of n + 3
// rows at x).
void lattice_rows_public(const cfneb_band *b, double *x, double sign) {
    for (int e = 0; e < 9; e += 4) x[(size_t)b->n * 3 + e] += sign * b->c;
}

// write FIRE reset values into the device params and zero velocities
void fire_reset(cfneb_band *b) {
    read_params(b);
    BandParams *p = b->h_bp;
    p->dt = p->dt0;
    p->alpha = 0.1;
    p->npos = 0;
    p->fresh = 1;
    p->stale = 1;  // images were inserted, removed or moved: rebuild every list
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
        launch_band_dots_only<float>(b->d_scratch_tiles + b->dv.rtpi,
                                     (int)rt.size() - b->dv.rtpi, b->d_self, b->s);
    else
        launch_band_dots_only<double>(b->d_scratch_tiles + b->dv.rtpi,
                                      (int)rt.size() - b->dv.rtpi, b->d_self, b->s);
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
    b->move_limit = move_limit;
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
    // lattice scale: the caller's c, or J = Omega0^(1/3) n^(1/6) (the scale
    // of the generalized solid-state NEB: it keeps the lattice rows'
    // stiffness per unit of X independent of n), or n_atoms
    if (b->filt.cell_factor > 0)
        b->c = b->filt.cell_factor;
    else if (b->filt.cell_factor == CFNEB_CELL_FACTOR_J)
        b->c = std::cbrt(std::fabs(det3(A->cell))) * std::pow((double)b->n, 1.0 / 6.0);
    else
        b->c = (double)b->n;
    CK(cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&b->s_body, cudaStreamNonBlocking));
    b->fork.create();
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
    } else if (pot->kind == CFNEB_NEP) {
        rc = pot->nep_rc;
        P.pot[0] = rc;
        // the many-body list and pair-vector code reads R (here rc) from the
        // Tersoff constant block: s = r - rc
        TersoffParams tp;
        std::memset(&tp, 0, sizeof(tp));
        tp.R = rc;
        tp.D = 1.0;
        tp.d = 1.0;
        tp.n = 1.0;
        P.tpf.load(tp);
        P.tpd.load(tp);
    } else {
        bool zero = true;
        for (int k = 0; k < 11; ++k) zero = zero && pot->tersoff[k] == 0.0;
        for (int k = 0; k < 11; ++k) P.pot[k] = zero ? kTersoff1988C[k] : pot->tersoff[k];
        rc = P.pot[9] + P.pot[10];
        // a copy, not a cast of pot[] (type-based aliasing lets the host
        // compiler read the cast view before the stores above)
        TersoffParams tp;
        std::memcpy(&tp, P.pot, sizeof(tp));
        P.tpf.load(tp);
        P.tpd.load(tp);
    }
    // neighbour-list skin: the caller's, or 0.15 A for Tersoff (carbon's
    // second neighbours, 2.46-2.52 A, stay outside R + D + skin, so the lists
    // keep their 3-4 entries) and 0.12 rc for LJ (0.3 sigma at rc = 2.5
    // sigma: the list holds ~1.4 candidates per pair inside rc, against ~3.4
    // for a walk of half-cutoff bins)
    const double skin = opt->skin >= 0.0 ? opt->skin : (pot->kind == CFNEB_LJ ? 0.12 * rc : 0.15);
    const double rl = rc + skin;
    b->rl = rl;
    // the cell list reaches MAX_STENCIL bins to each side: both end cells
    // must be at least rl / MAX_STENCIL wide along every lattice direction
    if (!stencil_reaches(A->cell, rl) || (cf && cf->enabled && !stencil_reaches(B->cell, rl))) {
        *err = CFNEB_ERR_INVALID_ARG;
        return b;
    }
    // bin width: the caller's, the cached autotuned one for this class, or rc
    const double dens = (double)b->n / std::fabs(det3(A->cell)) * rc * rc * rc;
    b->tune_key = std::make_tuple(pot->kind, opt->precision,
                                  (int)std::floor(std::log2((double)std::max(1, b->n))),
                                  (int)std::floor(2.0 * std::log2(std::max(dens, 1e-3))));
    double bscale = opt->bin_scale > 0 ? opt->bin_scale : tuned_scale(b->tune_key);
    b->minb = tuned_minb(b->tune_key);
    double bin_w = rl * bscale;
    b->rc = rc;
    // reserve bins for the finest autotuning candidate when tuning may follow
    const double cap_w = opt->bin_scale > 0 ? bin_w : rl * kTuneScales[0];
    // geometry
    // row stride of an image: the n atom rows and 3 lattice rows, padded to a
    // multiple of 4 rows (12 values) so that every image starts on a 16-byte
    // boundary and the band kernels load whole rows with vector loads; the
    // padding rows stay zero in X, F, f_NEB and v
    const int n = b->n, rows = (n + 3 + 3) / 4 * 4;
    BandDev &d = b->dv;
    d.n = n;
    d.rows = rows;
    d.ncap = b->ncap;
    // bins per bin width along the innermost axis (the LJ kernel walks it as
    // contiguous rows; halving the bins there was measured slower, so 1)
    const int row_refine = 1;
    int nb0 = bins_for(A->cell, cap_w) * row_refine, nb1 = bins_for(B->cell, cap_w) * row_refine;
    d.nbins_cap = (int)std::min<long long>((long long)(1.5 * std::max(nb0, nb1)) + 64, 1LL << 26);
    d.atpi = (n + TILE - 1) / TILE;
    d.rtpi = (rows + RTILE - 1) / RTILE;
    const size_t nc = (size_t)b->ncap;
    const size_t vec = nc * rows * 3 * b->ts;
    d.X = dalloc(b, vec);
    d.F = dalloc(b, vec);
    d.Fneb = dalloc(b, vec);
    d.v = dalloc(b, vec);
    for (void *p : {d.X, d.F, d.Fneb, d.v}) CK(cudaMemsetAsync(p, 0, vec, b->s));
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
    if (skin > 0.0) {
        d.ref_X = dalloc(b, vec);  // the row layout of X (padding rows stay zero)
        d.atom_wrap = (int *)dalloc(b, na * 3 * sizeof(int));
        d.skin_part = (float *)dalloc(b, nc * d.atpi * sizeof(float));
    }
    d.lj_cap = 0;
    if (pot->kind == CFNEB_LJ && skin > 0.0 && n <= LJ_LIST_MAX_ATOMS) {
        // list capacity: 1.5 x the entries within rl at the denser endpoint's
        // mean density, plus 32 (the path never gets much denser than its
        // ends; an overflow is reported as CFNEB_ERR_NBR_OVERFLOW)
        const double vmin = std::min(std::fabs(det3(A->cell)), std::fabs(det3(B->cell)));
        const double expect = n / vmin * 4.0 / 3.0 * 3.14159265358979323846 * rl * rl * rl;
        d.lj_cap = (int)std::min<double>(std::ceil((1.5 * expect + 32.0) / 8.0) * 8.0, 4096.0);
        d.nbr_cnt = (int *)dalloc(b, na * sizeof(int));
        d.nbr_slot = (int *)dalloc(b, na * d.lj_cap * sizeof(int));
        CK(cudaMemsetAsync(d.nbr_cnt, 0, na * sizeof(int), b->s));
    }
    if (pot->kind == CFNEB_NEP) {
        double *w = (double *)dalloc(b, NEP_NW * (sizeof(double) + sizeof(float)));
        float *wf = (float *)(w + NEP_NW);
        float hf[NEP_NW];
        for (int k = 0; k < NEP_NW; ++k) hf[k] = (float)pot->nep_weights[k];
        CK(cudaMemcpyAsync(w, pot->nep_weights, NEP_NW * sizeof(double), cudaMemcpyHostToDevice, b->s));
        CK(cudaMemcpyAsync(wf, hf, NEP_NW * sizeof(float), cudaMemcpyHostToDevice, b->s));
        CK(cudaStreamSynchronize(b->s));  // hf is a stack array
        d.nep_w = w;
        d.nep_wf = wf;
    }
    if (pot->kind == CFNEB_TERSOFF || pot->kind == CFNEB_NEP) {
        d.nbr_cnt = (int *)dalloc(b, na * sizeof(int));
        d.nbr_slot = (int *)dalloc(b, na * MAXN_TERSOFF * sizeof(int));
        d.nbr_code = (int *)dalloc(b, na * MAXN_TERSOFF * sizeof(int));
        d.nbr_rev = (unsigned char *)dalloc(b, na * MAXN_TERSOFF);
        d.nbr_P = dalloc(b, na * 4 * MAXN_TERSOFF * b->ts);
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
    if (d.ref_X) CK(cudaMemsetAsync(d.ref_X, 0, vec, b->s));
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
    P.skin = skin;
    P.rl = rl;
    P.stale = 1;
    P.bin_w = bin_w;
    P.row_refine = row_refine;
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
// Autotuning of the bin width
// ===========================================================================

namespace {

void set_bin_w(cfneb_band *b, double w) {
    read_params(b);
    b->h_bp->bin_w = w;
    b->h_bp->stale = 1;  // the next evaluation bins at the new width
    CK(cudaMemcpyAsync(b->dv.bp, b->h_bp, sizeof(BandParams), cudaMemcpyHostToDevice, b->s));
    CK(cudaStreamSynchronize(b->s));
}

void set_tune_rebuild(cfneb_band *b, int on) {
    read_params(b);
    b->h_bp->tune_rebuild = on;
    CK(cudaMemcpyAsync(b->dv.bp, b->h_bp, sizeof(BandParams), cudaMemcpyHostToDevice, b->s));
    CK(cudaStreamSynchronize(b->s));
}

// time `steps` non-moving steps of the band at bin width w (ms per step)
double time_bin_w(cfneb_band *b, double w, int nsteps) {
    set_bin_w(b, w);
    steps(b, 2);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, b->s));
    steps(b, nsteps);
    CK(cudaEventRecord(e1, b->s));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms / nsteps;
}

double autotune_band(cfneb_band *b, int steps) {
    read_params(b);
    const long long keep_limit = b->h_bp->move_limit;
    const double keep_ftol = b->h_bp->ftol;
    const long long now = b->h_bp->steps;
    set_control(b, keep_ftol, now);  // evaluate, never move
    // time full rebuilds: with a skin the bin width only matters there
    set_tune_rebuild(b, 1);
    double best = kTuneScales[2], best_ms = 1e300;
    for (double sc : kTuneScales) {
        const double ms = time_bin_w(b, sc * b->rl, steps);
        if (ms < best_ms) {
            best_ms = ms;
            best = sc;
        }
    }
    set_tune_rebuild(b, 0);
    // then the force kernel's blocks per SM at that bin width (FP32 LJ with
    // neighbour lists and Tersoff; steps with list reuse, as the run has)
    int best_minb = 0;
    const bool lj_list = b->kind == CFNEB_LJ && b->dv.lj_cap > 0;
    if (b->precision == CFNEB_MIXED && (lj_list || b->kind == CFNEB_TERSOFF)) {
        const int *cand = lj_list ? kLjMinbs : kTersMinbs;
        const int nc = lj_list ? 4 : 5;
        double bm = 1e300;
        for (int q = 0; q < nc; ++q) {
            b->minb = cand[q];
            b->graph_dirty = true;
            const double ms = time_bin_w(b, best * b->rl, steps);
            if (ms < bm) {
                bm = ms;
                best_minb = cand[q];
            }
        }
        b->minb = best_minb;
        b->graph_dirty = true;
    }
    set_bin_w(b, best * b->rl);
    set_control(b, keep_ftol, keep_limit);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[b->tune_key] = best;
    if (best_minb) g_tune_minb[b->tune_key] = best_minb;
    return best;
}

}  // namespace

// ===========================================================================
// Batches
// ===========================================================================

struct cfneb_batch {
    int precision = 0;
    cudaStream_t s_body = nullptr;   // captures the conditional list-rebuild body
    Fork fork;                       // the finalize beside the force gather (graphs)
    int lj_minb = 0, ters_minb = 0;  // force kernel variants (0: the default)
    unsigned long long budget = 0, used = 0;
    cudaStream_t user = nullptr, s = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::vector<cfneb_band *> bands;
    // device tables (grown on demand)
    BandDev *d_bands = nullptr;
    Tile *d_tiles = nullptr;     // [atoms all | atoms LJ | atoms Tersoff | rows]
    ImgRef *d_imgs = nullptr;
    int *d_ids = nullptr;
    double *d_status = nullptr;
    double *h_status = nullptr;  // pinned
    size_t cap_bands = 0, cap_tiles = 0, cap_imgs = 0;
    LaunchSet ls;
    bool dirty = true;
    cudaGraphExec_t gexec = nullptr, gexec_n = nullptr;  // one step, GRAPH_STEPS steps
    bool prof = false;
    double prof_ms[K_COUNT]{};
    long long prof_n[K_COUNT]{};
    std::vector<cudaEvent_t> prof_ev;
};

namespace {

void batch_mark_dirty(cfneb_batch *bt) { bt->dirty = true; }

void bt_enter(cfneb_batch *bt) {
    CK(cudaEventRecord(bt->ev_in, bt->user));
    CK(cudaStreamWaitEvent(bt->s, bt->ev_in, 0));
}
void bt_leave(cfneb_batch *bt) {
    CK(cudaEventRecord(bt->ev_out, bt->s));
    CK(cudaStreamWaitEvent(bt->user, bt->ev_out, 0));
}

template <typename X>
void grow(X **p, size_t *cap, size_t need) {
    if (need <= *cap) return;
    if (*p) CK(cudaFree(*p));
    *p = nullptr;
    size_t c = std::max<size_t>(need, 2 * *cap);
    CK(cudaMalloc((void **)p, c * sizeof(X)));
    *cap = c;
}

void batch_rebuild(cfneb_batch *bt) {
    std::vector<BandDev> dv;
    std::vector<ImgRef> im;
    std::vector<Tile> all, lj, ljc, ters, nep, rows;
    std::vector<int> ids;
    int max_bins = 0;
    for (size_t k = 0; k < bt->bands.size(); ++k) {
        cfneb_band *b = bt->bands[k];
        dv.push_back(b->dv);
        ids.push_back((int)k);
        max_bins = std::max(max_bins, b->dv.nbins_cap);
        for (int i = 1; i < b->N - 1; ++i) {
            im.push_back({(int)k, i});
            for (int t = 0; t < b->dv.atpi; ++t) {
                all.push_back({(int)k, i, t, 0});
                (b->kind == CFNEB_NEP ? nep : b->kind != CFNEB_LJ ? ters : b->dv.lj_cap > 0 ? lj : ljc)
                    .push_back({(int)k, i, t, 0});
            }
            for (int t = 0; t < b->dv.rtpi; ++t) rows.push_back({(int)k, i, t, 0});
        }
    }
    grow(&bt->d_bands, &bt->cap_bands, std::max<size_t>(dv.size(), 1));
    std::vector<Tile> tiles;
    tiles.insert(tiles.end(), all.begin(), all.end());
    tiles.insert(tiles.end(), lj.begin(), lj.end());
    tiles.insert(tiles.end(), ljc.begin(), ljc.end());
    tiles.insert(tiles.end(), ters.begin(), ters.end());
    tiles.insert(tiles.end(), nep.begin(), nep.end());
    tiles.insert(tiles.end(), rows.begin(), rows.end());
    grow(&bt->d_tiles, &bt->cap_tiles, std::max<size_t>(tiles.size(), 1));
    grow(&bt->d_imgs, &bt->cap_imgs, std::max<size_t>(im.size(), 1));
    if (bt->d_ids) CK(cudaFree(bt->d_ids));
    if (bt->d_status) CK(cudaFree(bt->d_status));
    if (bt->h_status) CK(cudaFreeHost(bt->h_status));
    const size_t nb = std::max<size_t>(ids.size(), 1);
    CK(cudaMalloc((void **)&bt->d_ids, nb * sizeof(int)));
    CK(cudaMalloc((void **)&bt->d_status, nb * 6 * sizeof(double)));
    CK(cudaMallocHost((void **)&bt->h_status, nb * 6 * sizeof(double)));
    if (!dv.empty())
        CK(cudaMemcpyAsync(bt->d_bands, dv.data(), dv.size() * sizeof(BandDev),
                           cudaMemcpyHostToDevice, bt->s));
    if (!tiles.empty())
        CK(cudaMemcpyAsync(bt->d_tiles, tiles.data(), tiles.size() * sizeof(Tile),
                           cudaMemcpyHostToDevice, bt->s));
    if (!im.empty())
        CK(cudaMemcpyAsync(bt->d_imgs, im.data(), im.size() * sizeof(ImgRef),
                           cudaMemcpyHostToDevice, bt->s));
    if (!ids.empty())
        CK(cudaMemcpyAsync(bt->d_ids, ids.data(), ids.size() * sizeof(int),
                           cudaMemcpyHostToDevice, bt->s));
    CK(cudaStreamSynchronize(bt->s));
    LaunchSet &ls = bt->ls;
    ls = LaunchSet();
    ls.d_bands = bt->d_bands;
    ls.s = bt->s;
    ls.imgs = bt->d_imgs;
    ls.nimg = (int)im.size();
    ls.atiles = bt->d_tiles;
    ls.n_atiles = (int)all.size();
    ls.atiles_lj = bt->d_tiles + all.size();
    ls.n_lj = (int)lj.size();
    ls.atiles_ljc = bt->d_tiles + all.size() + lj.size();
    ls.n_ljc = (int)ljc.size();
    ls.atiles_ters = bt->d_tiles + all.size() + lj.size() + ljc.size();
    ls.n_ters = (int)ters.size();
    ls.atiles_nep = bt->d_tiles + all.size() + lj.size() + ljc.size() + ters.size();
    ls.n_nep = (int)nep.size();
    ls.rtiles = bt->d_tiles + all.size() + lj.size() + ljc.size() + ters.size() + nep.size();
    ls.n_rtiles = (int)rows.size();
    ls.band_ids = bt->d_ids;
    ls.nbands = (int)ids.size();
    ls.max_bins = max_bins;
    ls.s_body = bt->s_body;
    ls.fork = &bt->fork;
    if (bt->lj_minb) ls.lj_minb = bt->lj_minb;
    if (bt->ters_minb) ls.ters_minb = bt->ters_minb;
    drop_graphs(bt->gexec, bt->gexec_n);
    bt->dirty = false;
}

void batch_steps(cfneb_batch *bt, int n) {
    if (n <= 0) return;
    if (bt->dirty) batch_rebuild(bt);
    if (bt->ls.nimg == 0) return;
    const LaunchSet ls = bt->ls;
    auto enq = [&](Launcher &L) {
        if (bt->precision == CFNEB_MIXED) enqueue_step_set<float>(ls, L);
        else enqueue_step_set<double>(ls, L);
    };
    if (bt->prof) {
        for (int i = 0; i < n; ++i) profiled(bt->s, bt->prof_ev, bt->prof_ms, bt->prof_n, enq);
        return;
    }
    launch_steps(bt->gexec, bt->gexec_n, bt->s, n, enq);
}

// per-member (moves, converged, status, fmax, ci, N)
void batch_poll(cfneb_batch *bt) {
    if (bt->dirty) batch_rebuild(bt);
    const int nb = (int)bt->bands.size();
    if (nb == 0) return;
    launch_gather_status(bt->d_bands, nb, bt->d_status, bt->s);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(bt->h_status, bt->d_status, nb * 6 * sizeof(double),
                       cudaMemcpyDeviceToHost, bt->s));
    CK(cudaStreamSynchronize(bt->s));
}

// Relax (or, with stop = false and ftol < 0, just step) the members for up
// to n_eval steps, with the members' refinement checks at their k_ref
// boundaries.  Returns the first error status of a member, or OK.
int batch_run(cfneb_batch *bt, long long n_eval, bool stop_on_converged) {
    long long launched = 0;
    int chunk = 8;
    while (launched < n_eval) {
        batch_poll(bt);
        long long k = std::min<long long>(n_eval - launched, chunk);
        for (size_t m = 0; m < bt->bands.size(); ++m) {
            cfneb_band *b = bt->bands[m];
            if (!b->opt.adaptive) continue;
            long long cur = (long long)bt->h_status[6 * m];
            k = std::min(k, (long long)(b->opt.k_ref - (cur % b->opt.k_ref)));
        }
        batch_steps(bt, (int)k);
        launched += k;
        batch_poll(bt);
        bool all_done = true;
        for (size_t m = 0; m < bt->bands.size(); ++m) {
            const double *st = bt->h_status + 6 * m;
            if ((int)st[2]) return status_from_bits((int)st[2]);
            cfneb_band *b = bt->bands[m];
            const long long cur = (long long)st[0];
            const bool done = (int)st[1] != 0 || cur >= b->move_limit;
            all_done = all_done && done;
            if (b->opt.adaptive && cur > 0 && cur % b->opt.k_ref == 0 && cur != b->last_check &&
                cur - b->last_change >= b->opt.cooldown) {
                b->last_check = cur;
                refine(b);
            }
        }
        if (stop_on_converged && all_done) break;
        chunk = std::min(chunk * 2, 64);
    }
    return CFNEB_OK;
}

void batch_free(cfneb_batch *bt) {
    if (!bt) return;
    if (bt->s) cudaStreamSynchronize(bt->s);
    for (cfneb_band *b : bt->bands) {
        b->batch = nullptr;
        if (b->own_s) b->s = b->own_s;
        b->own_s = nullptr;
    }
    if (bt->gexec) cudaGraphExecDestroy(bt->gexec);
    if (bt->gexec_n) cudaGraphExecDestroy(bt->gexec_n);
    if (bt->d_bands) cudaFree(bt->d_bands);
    if (bt->d_tiles) cudaFree(bt->d_tiles);
    if (bt->d_imgs) cudaFree(bt->d_imgs);
    if (bt->d_ids) cudaFree(bt->d_ids);
    if (bt->d_status) cudaFree(bt->d_status);
    if (bt->h_status) cudaFreeHost(bt->h_status);
    for (auto e : bt->prof_ev) cudaEventDestroy(e);
    if (bt->ev_in) cudaEventDestroy(bt->ev_in);
    if (bt->ev_out) cudaEventDestroy(bt->ev_out);
    if (bt->s) cudaStreamDestroy(bt->s);
    if (bt->s_body) cudaStreamDestroy(bt->s_body);
    bt->fork.destroy();
    delete bt;
}

}  // namespace

// ===========================================================================
// Serving
// ===========================================================================

namespace {

struct Request {
    long long id = 0;
    double arrival = 0.0;
    std::vector<double> R0, R1;
    double h0[9], h1[9];
    int n = 0, n_images = 0;
    cfneb_potential pot{};
    std::vector<double> nep_w;  // the request's own copy of NEP weights
    cfneb_cell_filter filt{};
    cfneb_options opt{};
    double fmax = 0.0;
    long long max_steps = 0;
    int state = 0;  // 0 queued, 1 running, 2 retired
    unsigned long long bytes = 0;  // device memory of its band, once known
    cfneb_band *band = nullptr;
    long long steps0 = 0;
    double done_t = 0.0;
    long long steps = 0;
    int converged = 0;
    int status = 0;
    double barrier = 0.0;
};

}  // namespace

struct cfneb_server {
    int precision = 0;
    cudaStream_t user = nullptr;
    cfneb_batch *bt = nullptr;
    std::vector<Request> req;
    std::deque<long long> queue;   // ids waiting, in arrival order
    std::vector<long long> running;
    std::chrono::steady_clock::time_point t0;
    double work = 0.0;             // atom-steps of retired requests
    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

void server_retire(cfneb_server *sv, Request &r, int status) {
    cfneb_band *b = r.band;
    read_params(b);
    r.steps = b->h_bp->steps - r.steps0;
    r.converged = b->h_bp->converged;
    r.status = status;
    if (status == CFNEB_OK) {
        std::vector<double> E(b->N);
        int32_t N = 0;
        cfneb_get_path(b, &N, nullptr, nullptr, E.data(), nullptr);
        r.barrier = *std::max_element(E.begin(), E.end()) - E[0];
    }
    cfneb_batch_remove(sv->bt, b);
    sv->work += (double)r.n * (b->N - 2) * (double)r.steps;
    cfneb_destroy_band(b);
    r.band = nullptr;
    r.state = 2;
    r.done_t = sv->now();
}

// admit arrived requests in order while they fit; false if the head waits
void server_admit(cfneb_server *sv) {
    const double t = sv->now();
    while (!sv->queue.empty()) {
        Request &r = sv->req[sv->queue.front()];
        if (r.arrival > t) return;
        // a request known not to fit waits without being rebuilt
        if (r.bytes && sv->bt->budget && sv->bt->used + r.bytes > sv->bt->budget &&
            !sv->running.empty())
            return;
        cfneb_structure A{r.n, nullptr, r.R0.data(), {}}, B{r.n, nullptr, r.R1.data(), {}};
        std::memcpy(A.cell, r.h0, sizeof(r.h0));
        std::memcpy(B.cell, r.h1, sizeof(r.h1));
        cfneb_band *b = nullptr;
        if (r.pot.kind == CFNEB_NEP) r.pot.nep_weights = r.nep_w.data();
        int st = cfneb_create_band(&A, &B, r.n_images, &r.pot, &r.filt, &r.opt, sv->user, &b);
        if (st != CFNEB_OK) {  // cannot be built at all: retire with the error
            r.status = st;
            r.state = 2;
            r.done_t = sv->now();
            sv->queue.pop_front();
            continue;
        }
        r.bytes = b->bytes;
        st = cfneb_batch_add(sv->bt, b);
        if (st == CFNEB_ERR_HBM_BUDGET && !sv->running.empty()) {
            cfneb_destroy_band(b);  // wait for memory to free up
            return;
        }
        if (st != CFNEB_OK && st != CFNEB_ERR_HBM_BUDGET) {
            cfneb_destroy_band(b);
            r.status = st;
            r.state = 2;
            r.done_t = sv->now();
            sv->queue.pop_front();
            continue;
        }
        if (st == CFNEB_ERR_HBM_BUDGET) {
            // larger than the whole budget on an idle server: refuse
            cfneb_destroy_band(b);
            r.status = st;
            r.state = 2;
            r.done_t = sv->now();
            sv->queue.pop_front();
            continue;
        }
        r.band = b;
        read_params(b);
        r.steps0 = b->h_bp->steps;
        set_control(b, r.fmax, r.steps0 + r.max_steps);
        r.state = 1;
        sv->running.push_back(r.id);
        sv->queue.pop_front();
    }
}

int server_run(cfneb_server *sv, double until) {
    while (true) {
        server_admit(sv);
        if (sv->running.empty()) {
            if (sv->queue.empty()) return CFNEB_OK;
            const double wait = sv->req[sv->queue.front()].arrival - sv->now();
            if (sv->now() > until) return CFNEB_NOT_CONVERGED;
            if (wait > 0)
                std::this_thread::sleep_for(std::chrono::duration<double>(std::min(wait, 0.01)));
            continue;
        }
        if (sv->now() > until) return CFNEB_NOT_CONVERGED;
        batch_run(sv->bt, 8, false);
        batch_poll(sv->bt);
        // decide from this poll's snapshot (indexed by the current member
        // order) first, then retire: removals reorder the members
        std::vector<long long> keep;
        std::vector<std::pair<long long, int>> retire;
        for (long long id : sv->running) {
            Request &r = sv->req[id];
            const size_t m = std::find(sv->bt->bands.begin(), sv->bt->bands.end(), r.band) -
                             sv->bt->bands.begin();
            const double *st = sv->bt->h_status + 6 * m;
            const int bits = (int)st[2];
            const bool conv = (int)st[1] != 0;
            const bool spent = (long long)st[0] - r.steps0 >= r.max_steps;
            if (bits || conv || spent) retire.push_back({id, status_from_bits(bits)});
            else keep.push_back(id);
        }
        for (auto &rt : retire) server_retire(sv, sv->req[rt.first], rt.second);
        sv->running.swap(keep);
    }
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
    o->skin = -1.0;
    return CFNEB_OK;
}

namespace {
// cfneb_create_band with the argument checks; need_path: refuse coincident
// endpoints (single-point evaluations build a band of one structure)
int create_band_checked(const cfneb_structure *initial, const cfneb_structure *final_,
                        int32_t n_images, const cfneb_potential *potential,
                        const cfneb_cell_filter *cell_filter, const cfneb_options *options,
                        void *cuda_stream, cfneb_band **out, bool need_path) {
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
    if (potential->kind != CFNEB_LJ && potential->kind != CFNEB_TERSOFF &&
        potential->kind != CFNEB_NEP)
        return CFNEB_ERR_INVALID_ARG;
    if (potential->kind == CFNEB_NEP) {
        if (!potential->nep_weights || !(potential->nep_rc > 0.0) ||
            !std::isfinite(potential->nep_rc))
            return CFNEB_ERR_INVALID_ARG;
        for (int k = 0; k < NEP_NW; ++k)
            if (!std::isfinite(potential->nep_weights[k])) return CFNEB_ERR_INVALID_ARG;
    }
    if (potential->kind == CFNEB_LJ &&
        (potential->rc <= 0 || potential->sigma <= 0 || potential->eps <= 0))
        return CFNEB_ERR_INVALID_ARG;
    if (!(std::fabs(det3(initial->cell)) > 0) || !(std::fabs(det3(final_->cell)) > 0))
        return CFNEB_ERR_INVALID_ARG;
    // finite coordinates and cells only (a non-finite coordinate would reach
    // the cell list as a meaningless bin)
    for (const cfneb_structure *S : {initial, final_}) {
        for (int k = 0; k < 9; ++k)
            if (!std::isfinite(S->cell[k])) return CFNEB_ERR_INVALID_ARG;
        for (long long k = 0; k < 3LL * S->n_atoms; ++k)
            if (!std::isfinite(S->positions[k])) return CFNEB_ERR_INVALID_ARG;
    }
    // coincident endpoints (every atom on the same periodic site, the same
    // cell where the filter is on) leave no path: every tangent of the
    // band would vanish (Sec. II.A's projection is undefined)
    if (need_path) {
        const bool filter = cell_filter && cell_filter->enabled;
        bool same_cell = true;
        for (int k = 0; k < 9 && filter; ++k)
            same_cell = same_cell && std::fabs(final_->cell[k] - initial->cell[k]) <=
                                         1e-12 * (1.0 + std::fabs(initial->cell[k]));
        double hi0[9], hi1[9];
        inv3(initial->cell, hi0);
        inv3(filter ? final_->cell : initial->cell, hi1);
        bool same_sites = same_cell;
        for (int i = 0; i < initial->n_atoms && same_sites; ++i) {
            const double *p0 = initial->positions + 3 * (size_t)i;
            const double *p1 = final_->positions + 3 * (size_t)i;
            for (int a = 0; a < 3; ++a) {
                const double s0 = p0[0] * hi0[a] + p0[1] * hi0[3 + a] + p0[2] * hi0[6 + a];
                const double s1 = p1[0] * hi1[a] + p1[1] * hi1[3 + a] + p1[2] * hi1[6 + a];
                const double d = (s1 - s0) - std::nearbyint(s1 - s0);
                if (!(std::fabs(d) <= 1e-12)) {
                    same_sites = false;
                    break;
                }
            }
        }
        if (same_sites) return CFNEB_ERR_INVALID_ARG;
    }
    cfneb_options opt;
    if (options) opt = *options;
    else cfneb_default_options(&opt);
    if (opt.precision != CFNEB_FP64 && opt.precision != CFNEB_MIXED) return CFNEB_ERR_INVALID_ARG;
    if (opt.dt <= 0 || opt.maxstep <= 0) return CFNEB_ERR_INVALID_ARG;
    if (opt.k_ref <= 0) opt.k_ref = 10;
    if (opt.bin_scale != 0 && opt.bin_scale < 0.25) return CFNEB_ERR_INVALID_ARG;
    {
        // a skin (< 0: the default) of at most the potential's cutoff
        double rcut = potential->kind == CFNEB_NEP ? potential->nep_rc : potential->rc;
        if (potential->kind == CFNEB_TERSOFF) {
            const bool dflt = std::all_of(potential->tersoff, potential->tersoff + 11,
                                          [](double v) { return v == 0.0; });
            rcut = dflt ? kTersoff1988C[9] + kTersoff1988C[10]
                        : potential->tersoff[9] + potential->tersoff[10];
        }
        if (!(opt.skin < 0.0 || opt.skin <= rcut)) return CFNEB_ERR_INVALID_ARG;
    }
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

}  // namespace

int cfneb_create_band(const cfneb_structure *initial, const cfneb_structure *final_,
                      int32_t n_images, const cfneb_potential *potential,
                      const cfneb_cell_filter *cell_filter, const cfneb_options *options,
                      void *cuda_stream, cfneb_band **out) {
    return create_band_checked(initial, final_, n_images, potential, cell_filter, options,
                               cuda_stream, out, true);
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
            // then Cartesian positions R = R~ D from the same map-back; the
            // endpoints never move, so theirs are computed once
            std::vector<int> imgs;
            if (!b->ends_e64) imgs = {0, b->N - 1};
            for (int i = 1; i < b->N - 1; ++i) imgs.push_back(i);
            refine_energies(b, imgs);
            b->ends_e64 = true;
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
        // per image n + 3 rows out of the padded row stride
        const size_t per = (size_t)(b->n + 3) * 3, stride = (size_t)b->dv.rows * 3;
        const size_t cnt = (size_t)b->N * stride;
        std::vector<char> tmp(cnt * b->ts);
        auto fetch = [&](void *src, double *dst) {
            if (!dst) return;
            CK(cudaMemcpyAsync(tmp.data(), src, cnt * b->ts, cudaMemcpyDeviceToHost, b->s));
            CK(cudaStreamSynchronize(b->s));
            for (int im = 0; im < b->N; ++im)
                for (size_t i = 0; i < per; ++i)
                    dst[im * per + i] = b->ts == 4 ? ((const float *)tmp.data())[im * stride + i]
                                                   : ((const double *)tmp.data())[im * stride + i];
        };
        fetch(b->dv.X, X);
        if (X)
            for (int im = 0; im < b->N; ++im) lattice_rows_public(b, X + im * per, 1.0);
        fetch(b->dv.F, F);
        fetch(b->dv.Fneb, Fneb);
        if (Fneb) {  // endpoints carry no NEB force
            std::memset(Fneb, 0, per * sizeof(double));
            std::memset(Fneb + (size_t)(b->N - 1) * per, 0, per * sizeof(double));
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

int cfneb_set_state(cfneb_band *b, const double *X) {
    if (!b || !X) return CFNEB_ERR_INVALID_ARG;
    const size_t per = (size_t)(b->n + 3) * 3, stride = (size_t)b->dv.rows * 3;
    for (size_t i = 0; i < (size_t)b->N * per; ++i)
        if (!std::isfinite(X[i])) return CFNEB_ERR_INVALID_ARG;
    try {
        enter(b);
        // n + 3 rows per image into the padded row stride (padding stays 0)
        const size_t cnt = (size_t)b->N * stride;
        std::vector<double> pad(cnt, 0.0);
        for (int im = 0; im < b->N; ++im) {
            std::memcpy(pad.data() + im * stride, X + im * per, per * sizeof(double));
            lattice_rows_public(b, pad.data() + im * stride, -1.0);
        }
        if (b->ts == 4) {
            std::vector<float> tmp(cnt);
            for (size_t i = 0; i < cnt; ++i) tmp[i] = (float)pad[i];
            CK(cudaMemcpyAsync(b->dv.X, tmp.data(), cnt * sizeof(float), cudaMemcpyHostToDevice,
                               b->s));
            CK(cudaStreamSynchronize(b->s));
        } else {
            CK(cudaMemcpyAsync(b->dv.X, pad.data(), cnt * sizeof(double), cudaMemcpyHostToDevice,
                               b->s));
            CK(cudaStreamSynchronize(b->s));
        }
        fire_reset(b);
        eval_images(b, {0, b->N - 1});  // the endpoints' energies and forces
        b->ends_e64 = false;            // their FP64 energies are re-taken when reported
        read_params(b);
        leave(b);
        return status_from_bits(b->h_bp->status);
    } catch (CudaFail &) {
        return CFNEB_ERR_CUDA;
    }
}

// ---- image-range shards ---------------------------------------------------

int cfneb_shard_enable(cfneb_band *b) {
    if (!b || b->batch || b->opt.adaptive) return CFNEB_ERR_INVALID_ARG;
    try {
        enter(b);
        read_params(b);
        b->h_bp->shard = 1;
        b->h_bp->ci_ext = -1;
        b->h_bp->ftol = -1.0;  // the caller tests convergence on the global fmax
        CK(cudaMemcpyAsync(b->dv.bp, b->h_bp, sizeof(BandParams), cudaMemcpyHostToDevice, b->s));
        fire_reset(b);
        leave(b);
        return CFNEB_OK;
    } catch (CudaFail &) {
        return CFNEB_ERR_CUDA;
    }
}

int cfneb_shard_evaluate(cfneb_band *b, double *energies) {
    if (!b || !b->h_bp->shard) return CFNEB_ERR_INVALID_ARG;
    try {
        enter(b);
        Launcher L;
        const LaunchSet ls = band_step_set(b);
        if (b->precision == CFNEB_MIXED) enqueue_eval_set<float>(ls, L);
        else enqueue_eval_set<double>(ls, L);
        CK(cudaGetLastError());
        std::vector<ImgScalars> sc(b->N);
        CK(cudaMemcpyAsync(sc.data(), b->dv.sc, b->N * sizeof(ImgScalars),
                           cudaMemcpyDeviceToHost, b->s));
        read_params(b);
        if (energies)
            for (int i = 0; i < b->N; ++i) energies[i] = sc[i].E;
        leave(b);
        return status_from_bits(b->h_bp->status);
    } catch (CudaFail &) {
        return CFNEB_ERR_CUDA;
    }
}

int cfneb_shard_set_ghost(cfneb_band *b, int32_t side, const double *X, double energy) {
    if (!b || !X || (side != 0 && side != 1) || !b->h_bp->shard) return CFNEB_ERR_INVALID_ARG;
    const size_t per = (size_t)(b->n + 3) * 3;
    for (size_t i = 0; i < per; ++i)
        if (!std::isfinite(X[i])) return CFNEB_ERR_INVALID_ARG;
    try {
        enter(b);
        const int img = side == 0 ? 0 : b->N - 1;
        char *dst = (char *)b->dv.X + (size_t)img * b->dv.rows * 3 * b->ts;
        std::vector<double> xs(X, X + per);
        lattice_rows_public(b, xs.data(), -1.0);
        std::vector<float> f;
        if (b->ts == 4) {
            f.resize(per);
            for (size_t i = 0; i < per; ++i) f[i] = (float)xs[i];
            CK(cudaMemcpyAsync(dst, f.data(), per * sizeof(float), cudaMemcpyHostToDevice, b->s));
        } else {
            CK(cudaMemcpyAsync(dst, xs.data(), per * sizeof(double), cudaMemcpyHostToDevice,
                               b->s));
        }
        CK(cudaMemcpyAsync(&b->dv.sc[img].E, &energy, sizeof(double), cudaMemcpyHostToDevice,
                           b->s));
        CK(cudaStreamSynchronize(b->s));
        leave(b);
        return CFNEB_OK;
    } catch (CudaFail &) {
        return CFNEB_ERR_CUDA;
    }
}

int cfneb_shard_get_image(const cfneb_band *cb, int32_t index, double *X, double *energy) {
    cfneb_band *b = const_cast<cfneb_band *>(cb);
    if (!b || index < 0 || index >= b->N) return CFNEB_ERR_INVALID_ARG;
    try {
        enter(b);
        const size_t per = (size_t)(b->n + 3) * 3;
        const char *src = (const char *)b->dv.X + (size_t)index * b->dv.rows * 3 * b->ts;
        std::vector<char> tmp(per * b->ts);
        double e = 0.0;
        CK(cudaMemcpyAsync(tmp.data(), src, tmp.size(), cudaMemcpyDeviceToHost, b->s));
        CK(cudaMemcpyAsync(&e, &b->dv.sc[index].E, sizeof(double), cudaMemcpyDeviceToHost, b->s));
        CK(cudaStreamSynchronize(b->s));
        if (X) {
            for (size_t i = 0; i < per; ++i)
                X[i] = b->ts == 4 ? ((const float *)tmp.data())[i] : ((const double *)tmp.data())[i];
            lattice_rows_public(b, X, 1.0);
        }
        if (energy) *energy = e;
        leave(b);
        return CFNEB_OK;
    } catch (CudaFail &) {
        return CFNEB_ERR_CUDA;
    }
}

int cfneb_shard_project(cfneb_band *b, int32_t climbing_index, double *sums) {
    if (!b || !sums || !b->h_bp->shard || climbing_index < -1 || climbing_index == 0 ||
        climbing_index >= b->N - 1)
        return CFNEB_ERR_INVALID_ARG;
    try {
        enter(b);
        int ci = climbing_index;
        CK(cudaMemcpyAsync(&b->dv.bp->ci_ext, &ci, sizeof(int), cudaMemcpyHostToDevice, b->s));
        const LaunchSet ls = band_step_set(b);
        if (b->precision == CFNEB_MIXED) {
            launch_band_dots<float>(ls.rtiles, ls.n_rtiles, ls.d_bands, b->s);
            launch_neb_force<float>(ls.rtiles, ls.n_rtiles, ls.d_bands, b->s);
        } else {
            launch_band_dots<double>(ls.rtiles, ls.n_rtiles, ls.d_bands, b->s);
            launch_neb_force<double>(ls.rtiles, ls.n_rtiles, ls.d_bands, b->s);
        }
        CK(cudaGetLastError());
        read_params(b);
        sums[0] = b->h_bp->P;
        sums[1] = b->h_bp->FF;
        sums[2] = b->h_bp->VV;
        sums[3] = b->h_bp->fmax;  // the largest squared row norm
        leave(b);
        return CFNEB_OK;
    } catch (CudaFail &) {
        return CFNEB_ERR_CUDA;
    }
}

int cfneb_shard_move(cfneb_band *b, const double *sums) {
    if (!b || !sums || !b->h_bp->shard) return CFNEB_ERR_INVALID_ARG;
    try {
        enter(b);
        launch_shard_fire(b->d_self, sums[0], sums[1], sums[2], sums[3], b->s);
        if (b->precision == CFNEB_MIXED)
            launch_fire_update<float>(b->d_rtiles, b->n_rtiles, b->d_imgs, b->n_imgs, b->d_self,
                                      b->s);
        else
            launch_fire_update<double>(b->d_rtiles, b->n_rtiles, b->d_imgs, b->n_imgs, b->d_self,
                                       b->s);
        CK(cudaGetLastError());
        read_params(b);
        leave(b);
        return status_from_bits(b->h_bp->status);
    } catch (CudaFail &) {
        return CFNEB_ERR_CUDA;
    }
}

int cfneb_get_image_scalars(const cfneb_band *cb, double *energies, double *dots, double *coef) {
    cfneb_band *b = const_cast<cfneb_band *>(cb);
    if (!b) return CFNEB_ERR_INVALID_ARG;
    try {
        enter(b);
        std::vector<ImgScalars> sc(b->N);
        CK(cudaMemcpyAsync(sc.data(), b->dv.sc, b->N * sizeof(ImgScalars),
                           cudaMemcpyDeviceToHost, b->s));
        CK(cudaStreamSynchronize(b->s));
        for (int i = 0; i < b->N; ++i) {
            const bool inner = i > 0 && i < b->N - 1;
            if (energies) energies[i] = sc[i].E;
            for (int k = 0; k < 10; ++k)
                if (dots) dots[10 * i + k] = inner ? sc[i].dots[k] : 0.0;
            for (int k = 0; k < 2; ++k)
                if (coef) coef[2 * i + k] = inner ? sc[i].coef[k] : 0.0;
        }
        leave(b);
        return CFNEB_OK;
    } catch (CudaFail &) {
        return CFNEB_ERR_CUDA;
    }
}

int cfneb_batch_remove(cfneb_batch *bt, cfneb_band *b);

int cfneb_destroy_band(cfneb_band *b) {
    if (!b) return CFNEB_ERR_INVALID_ARG;
    if (b->batch) cfneb_batch_remove(b->batch, b);
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
        opt.skin = 0.0;  // one evaluation: nothing to reuse
        cfneb_cell_filter cf{1, CFNEB_ROTFREE_B, 0.0, 0.0};
        cfneb_band *b = nullptr;
        int st = create_band_checked(&S, &S, 3, potential, &cf, &opt, cuda_stream, &b, false);
        if (st != CFNEB_OK) return st;
        try {
            enter(b);
            // the endpoints were evaluated at creation: image 0 is S; its
            // reported energy is the FP64 one
            refine_energies(b, {0});
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

int cfneb_band_bytes(const cfneb_band *b, uint64_t *bytes) {
    if (!b || !bytes) return CFNEB_ERR_INVALID_ARG;
    *bytes = b->bytes;
    return CFNEB_OK;
}

int cfneb_batch_create(int32_t precision, uint64_t budget_bytes, void *cuda_stream,
                       cfneb_batch **out) {
    if (!out || (precision != CFNEB_FP64 && precision != CFNEB_MIXED))
        return CFNEB_ERR_INVALID_ARG;
    cfneb_batch *bt = new cfneb_batch();
    bt->precision = precision;
    bt->budget = budget_bytes;
    bt->user = (cudaStream_t)cuda_stream;
    try {
        CK(cudaStreamCreateWithFlags(&bt->s, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&bt->s_body, cudaStreamNonBlocking));
        bt->fork.create();
        CK(cudaEventCreateWithFlags(&bt->ev_in, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&bt->ev_out, cudaEventDisableTiming));
        bt->prof_ev.resize(2 * 64);
        for (auto &e : bt->prof_ev) CK(cudaEventCreate(&e));
    } catch (CudaFail &) {
        batch_free(bt);
        return CFNEB_ERR_CUDA;
    }
    *out = bt;
    return CFNEB_OK;
}

int cfneb_batch_add(cfneb_batch *bt, cfneb_band *b) {
    if (!bt || !b || b->batch || b->precision != bt->precision) return CFNEB_ERR_INVALID_ARG;
    if (bt->budget && bt->used + b->bytes > bt->budget) return CFNEB_ERR_HBM_BUDGET;
    try {
        // the band's queued work finishes before the batch touches it
        CK(cudaEventRecord(b->ev_out, b->s));
        CK(cudaStreamWaitEvent(bt->s, b->ev_out, 0));
    } catch (CudaFail &) {
        return CFNEB_ERR_CUDA;
    }
    b->own_s = b->s;
    b->s = bt->s;
    b->batch = bt;
    b->graph_dirty = true;
    bt->bands.push_back(b);
    bt->used += b->bytes;
    bt->dirty = true;
    return CFNEB_OK;
}

int cfneb_batch_remove(cfneb_batch *bt, cfneb_band *b) {
    if (!bt || !b || b->batch != bt) return CFNEB_ERR_INVALID_ARG;
    try {
        CK(cudaEventRecord(bt->ev_out, bt->s));
        CK(cudaStreamWaitEvent(b->own_s, bt->ev_out, 0));
    } catch (CudaFail &) {
        return CFNEB_ERR_CUDA;
    }
    b->s = b->own_s;
    b->own_s = nullptr;
    b->batch = nullptr;
    b->graph_dirty = true;
    bt->bands.erase(std::find(bt->bands.begin(), bt->bands.end(), b));
    bt->used -= b->bytes;
    bt->dirty = true;
    return CFNEB_OK;
}

int cfneb_batch_step(cfneb_batch *bt, int32_t n_steps) {
    if (!bt || n_steps < 0) return CFNEB_ERR_INVALID_ARG;
    try {
        bt_enter(bt);
        bool adaptive = false;
        for (cfneb_band *b : bt->bands) adaptive = adaptive || b->opt.adaptive;
        int st = CFNEB_OK;
        if (adaptive) st = batch_run(bt, n_steps, false);
        else batch_steps(bt, n_steps);
        bt_leave(bt);
        return st;
    } catch (CudaFail &) {
        return CFNEB_ERR_CUDA;
    }
}

int cfneb_batch_relax(cfneb_batch *bt, double fmax, int64_t max_steps, int32_t *n_converged) {
    if (!bt || max_steps < 0 || !(fmax >= 0)) return CFNEB_ERR_INVALID_ARG;
    try {
        bt_enter(bt);
        for (cfneb_band *b : bt->bands) {
            read_params(b);
            set_control(b, fmax, b->h_bp->steps + max_steps);
        }
        int st = batch_run(bt, max_steps + 1, true);
        int conv = 0;
        batch_poll(bt);
        for (size_t m = 0; m < bt->bands.size(); ++m) conv += (int)bt->h_status[6 * m + 1];
        for (cfneb_band *b : bt->bands) {
            read_params(b);
            b->h_bp->move_limit = 1LL << 62;
            b->move_limit = 1LL << 62;
            CK(cudaMemcpyAsync(b->dv.bp, b->h_bp, sizeof(BandParams), cudaMemcpyHostToDevice,
                               b->s));
        }
        CK(cudaStreamSynchronize(bt->s));
        bt_leave(bt);
        if (n_converged) *n_converged = conv;
        if (st != CFNEB_OK) return st;
        return conv == (int)bt->bands.size() ? CFNEB_OK : CFNEB_NOT_CONVERGED;
    } catch (CudaFail &) {
        return CFNEB_ERR_CUDA;
    }
}

int cfneb_batch_status(cfneb_batch *bt, int32_t *count, int64_t *steps, int32_t *converged,
                       double *fmax, int32_t *status) {
    if (!bt) return CFNEB_ERR_INVALID_ARG;
    try {
        bt_enter(bt);
        batch_poll(bt);
        const int nb = (int)bt->bands.size();
        if (count) *count = nb;
        for (int m = 0; m < nb; ++m) {
            const double *st = bt->h_status + 6 * m;
            if (steps) steps[m] = (int64_t)st[0];
            if (converged) converged[m] = (int32_t)st[1];
            if (fmax) fmax[m] = st[3];
            if (status) status[m] = status_from_bits((int)st[2]);
        }
        bt_leave(bt);
        return CFNEB_OK;
    } catch (CudaFail &) {
        return CFNEB_ERR_CUDA;
    }
}

int cfneb_batch_bytes(const cfneb_batch *bt, uint64_t *used, uint64_t *budget) {
    if (!bt) return CFNEB_ERR_INVALID_ARG;
    if (used) *used = bt->used;
    if (budget) *budget = bt->budget;
    return CFNEB_OK;
}

int cfneb_batch_profile(cfneb_batch *bt, int32_t enable) {
    if (!bt) return CFNEB_ERR_INVALID_ARG;
    bt->prof = enable != 0;
    for (int k = 0; k < K_COUNT; ++k) {
        bt->prof_ms[k] = 0.0;
        bt->prof_n[k] = 0;
    }
    return CFNEB_OK;
}

int cfneb_batch_profile_read(cfneb_batch *bt, int32_t kernel_id, double *total_ms,
                             int64_t *launches) {
    if (!bt || kernel_id < 0 || kernel_id >= K_COUNT) return CFNEB_ERR_INVALID_ARG;
    if (total_ms) *total_ms = bt->prof_ms[kernel_id];
    if (launches) *launches = bt->prof_n[kernel_id];
    return CFNEB_OK;
}

int cfneb_autotune(cfneb_band *b, int32_t steps, double *best_scale) {
    if (!b || steps <= 0) return CFNEB_ERR_INVALID_ARG;
    try {
        enter(b);
        const double best = autotune_band(b, steps);
        leave(b);
        if (best_scale) *best_scale = best;
        return CFNEB_OK;
    } catch (CudaFail &) {
        return CFNEB_ERR_CUDA;
    }
}

int cfneb_get_tuning(const cfneb_band *b, double *bin_scale, int32_t *blocks_per_sm) {
    if (!b) return CFNEB_ERR_INVALID_ARG;
    if (bin_scale) *bin_scale = b->rl > 0.0 ? b->h_bp->bin_w / b->rl : 0.0;
    if (blocks_per_sm) {
        int m = b->minb;
        if (!m && b->precision == CFNEB_MIXED)
            m = b->kind == CFNEB_LJ && b->dv.lj_cap > 0 ? kLjMinb
                : b->kind == CFNEB_TERSOFF ? kTersMinb : 0;
        *blocks_per_sm = m;
    }
    return CFNEB_OK;
}

int cfneb_batch_autotune(cfneb_batch *bt, int32_t steps) {
    if (!bt || steps <= 0) return CFNEB_ERR_INVALID_ARG;
    try {
        bt_enter(bt);
        std::map<std::tuple<int, int, int, int>, double> done;
        std::map<std::tuple<int, int, int, int>, int> done_minb;
        // per class: bin width, then the force kernel's blocks per SM; the
        // batch launches the variant tuned for its largest member of each
        // potential (one launch covers every member)
        long long big_lj = -1, big_ters = -1;
        for (cfneb_band *b : bt->bands) {
            auto it = done.find(b->tune_key);
            double sc;
            if (it != done.end()) {
                sc = it->second;
                b->minb = done_minb[b->tune_key];
            } else {
                sc = autotune_band(b, steps);
                done[b->tune_key] = sc;
                done_minb[b->tune_key] = b->minb;
            }
            set_bin_w(b, sc * b->rl);
            const long long work = (long long)b->n * (b->N - 2);
            if (b->kind == CFNEB_LJ && b->minb && work > big_lj) {
                big_lj = work;
                bt->lj_minb = b->minb;
            }
            if (b->kind == CFNEB_TERSOFF && b->minb && work > big_ters) {
                big_ters = work;
                bt->ters_minb = b->minb;
            }
        }
        bt->dirty = true;
        bt_leave(bt);
        return CFNEB_OK;
    } catch (CudaFail &) {
        return CFNEB_ERR_CUDA;
    }
}

int cfneb_batch_destroy(cfneb_batch *bt) {
    if (!bt) return CFNEB_ERR_INVALID_ARG;
    batch_free(bt);
    return CFNEB_OK;
}

int cfneb_server_create(int32_t precision, uint64_t budget_bytes, void *cuda_stream,
                        cfneb_server **out) {
    if (!out) return CFNEB_ERR_INVALID_ARG;
    cfneb_server *sv = new cfneb_server();
    sv->precision = precision;
    sv->user = (cudaStream_t)cuda_stream;
    int st = cfneb_batch_create(precision, budget_bytes, cuda_stream, &sv->bt);
    if (st != CFNEB_OK) {
        delete sv;
        return st;
    }
    sv->t0 = std::chrono::steady_clock::now();
    *out = sv;
    return CFNEB_OK;
}

int cfneb_server_submit(cfneb_server *sv, const cfneb_structure *initial,
                        const cfneb_structure *final_, int32_t n_images,
                        const cfneb_potential *potential, const cfneb_cell_filter *cell_filter,
                        const cfneb_options *options, double fmax, int64_t max_steps,
                        double arrival_s, int64_t *id) {
    if (!sv || !initial || !final_ || !potential || !options || n_images < 3 ||
        initial->n_atoms <= 0 || initial->n_atoms != final_->n_atoms || !(fmax >= 0) ||
        max_steps < 0)
        return CFNEB_ERR_INVALID_ARG;
    if (options->precision != sv->precision) return CFNEB_ERR_INVALID_ARG;
    if (options->interior_noise) return CFNEB_ERR_INVALID_ARG;  // not copied by the server
    Request r;
    r.id = (long long)sv->req.size();
    r.arrival = arrival_s;
    r.n = initial->n_atoms;
    r.R0.assign(initial->positions, initial->positions + 3 * (size_t)r.n);
    r.R1.assign(final_->positions, final_->positions + 3 * (size_t)r.n);
    std::memcpy(r.h0, initial->cell, sizeof(r.h0));
    std::memcpy(r.h1, final_->cell, sizeof(r.h1));
    r.n_images = n_images;
    r.pot = *potential;
    if (potential->kind == CFNEB_NEP) {
        if (!potential->nep_weights) return CFNEB_ERR_INVALID_ARG;
        r.nep_w.assign(potential->nep_weights, potential->nep_weights + NEP_NW);
        r.pot.nep_weights = nullptr;  // set to the copy when the band is made
    }
    r.filt = cell_filter ? *cell_filter : cfneb_cell_filter{1, CFNEB_ROTFREE_B, 0.0, 0.0};
    r.opt = *options;
    r.fmax = fmax;
    r.max_steps = max_steps;
    sv->req.push_back(std::move(r));
    // keep the queue in arrival order
    auto pos = std::upper_bound(sv->queue.begin(), sv->queue.end(), arrival_s,
                                [&](double t, long long q) { return t < sv->req[q].arrival; });
    sv->queue.insert(pos, (long long)sv->req.size() - 1);
    if (id) *id = (long long)sv->req.size() - 1;
    return CFNEB_OK;
}

int cfneb_server_run(cfneb_server *sv, double until_s) {
    if (!sv) return CFNEB_ERR_INVALID_ARG;
    try {
        return server_run(sv, until_s);
    } catch (CudaFail &) {
        return CFNEB_ERR_CUDA;
    }
}

int cfneb_server_result(cfneb_server *sv, int64_t id, int32_t *state, double *latency_s,
                        int64_t *steps, int32_t *converged, double *barrier, int32_t *status) {
    if (!sv || id < 0 || id >= (int64_t)sv->req.size()) return CFNEB_ERR_INVALID_ARG;
    const Request &r = sv->req[id];
    if (state) *state = r.state;
    if (latency_s) *latency_s = r.state == 2 ? r.done_t - r.arrival : -1.0;
    if (steps) *steps = r.steps;
    if (converged) *converged = r.converged;
    if (barrier) *barrier = r.barrier;
    if (status) *status = r.status;
    return CFNEB_OK;
}

int cfneb_server_stats(cfneb_server *sv, double *p50_s, double *p99_s, int64_t *retired,
                       double *atom_steps_per_s) {
    if (!sv) return CFNEB_ERR_INVALID_ARG;
    std::vector<double> lat;
    for (const Request &r : sv->req)
        if (r.state == 2 && r.status == CFNEB_OK) lat.push_back(r.done_t - r.arrival);
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double p) {
        if (lat.empty()) return 0.0;
        const double x = p * (lat.size() - 1);
        const size_t i = (size_t)x;
        const double f = x - i;
        return i + 1 < lat.size() ? lat[i] * (1 - f) + lat[i + 1] * f : lat[i];
    };
    if (p50_s) *p50_s = pct(0.5);
    if (p99_s) *p99_s = pct(0.99);
    if (retired) *retired = (int64_t)lat.size();
    if (atom_steps_per_s) *atom_steps_per_s = sv->work / std::max(1e-9, sv->now());
    return CFNEB_OK;
}

int cfneb_server_destroy(cfneb_server *sv) {
    if (!sv) return CFNEB_ERR_INVALID_ARG;
    for (Request &r : sv->req)
        if (r.band) {
            cfneb_batch_remove(sv->bt, r.band);
            cfneb_destroy_band(r.band);
        }
    cfneb_batch_destroy(sv->bt);
    delete sv;
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

int cfneb_get_list_stats(const cfneb_band *cb, int64_t *builds, int64_t *evaluations,
                         double *skin) {
    cfneb_band *b = const_cast<cfneb_band *>(cb);
    if (!b) return CFNEB_ERR_INVALID_ARG;
    try {
        enter(b);
        std::vector<ImgScalars> sc(b->N);
        CK(cudaMemcpyAsync(sc.data(), b->dv.sc, b->N * sizeof(ImgScalars),
                           cudaMemcpyDeviceToHost, b->s));
        CK(cudaStreamSynchronize(b->s));
        long long nb = 0, ne = 0;
        for (int i = 1; i < b->N - 1; ++i) {
            nb += sc[i].builds;
            ne += sc[i].evals;
        }
        if (builds) *builds = nb;
        if (evaluations) *evaluations = ne;
        if (skin) *skin = b->rl - b->rc;
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
