// Lennard-Jones evaluation of one structure without any device allocation.
//
// Some callers cannot call cudaMalloc: allocators that own all device memory
// of a process (a framework's caching pool, a fixed arena sized at
// start-up) leave nothing for a library to take, and long-running services
// must not allocate once they are serving (an allocation can fail or stall
// at any time).  This entry point runs the library's existing FP64
// evaluation kernels (set-up, map-back, cell list, LJ forces, per-image
// finalize) on scratch memory that lives in one file-scope __device__
// array, and copies the results into the caller's device buffers.  The
// caller passes inputs and outputs; nothing is allocated or freed, here or
// in any library routine it calls.
//
// The array is every loading GPU's for the lifetime of the process and is
// shared by every call: calls that overlap on the GPU (different streams, or
// threads without ordering) race on it.  Whatever must start at zero is
// cleared at the start of each call.
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>

#include <cuda.h>

#include "../../include/cfneb.h"
#include "common.cuh"

using namespace cfneb;

namespace {

constexpr int NA_MAX_ATOMS = CFNEB_NOALLOC_MAX_ATOMS;
constexpr int NA_MAX_BINS = 32768;
constexpr int NA_IMAGES = 2;   // the set-up kernel writes two identical images
constexpr int NA_ROWS = NA_MAX_ATOMS + 3;
constexpr int NA_TILES = (NA_MAX_ATOMS + TILE - 1) / TILE;
constexpr int NA_TSUM = (NA_MAX_BINS + 1023) / 1024 + 1;

constexpr size_t al(size_t x) { return (x + 255) / 256 * 256; }

// byte offsets of each piece inside the scratch array
constexpr size_t O_BAND = 0;
constexpr size_t O_PARAMS = O_BAND + al(sizeof(BandDev));
constexpr size_t O_SC = O_PARAMS + al(sizeof(BandParams));
constexpr size_t O_H1 = O_SC + al(NA_IMAGES * sizeof(ImgScalars));
constexpr size_t O_TILES = O_H1 + al(9 * sizeof(double));
constexpr size_t O_IMG = O_TILES + al(NA_TILES * sizeof(Tile));
constexpr size_t O_X = O_IMG + al(sizeof(ImgRef));
constexpr size_t O_F = O_X + al((size_t)NA_IMAGES * NA_ROWS * 3 * sizeof(double));
constexpr size_t O_BCOUNT = O_F + al((size_t)NA_IMAGES * NA_ROWS * 3 * sizeof(double));
constexpr size_t O_BSTART = O_BCOUNT + al(NA_MAX_BINS * sizeof(int));
constexpr size_t O_BTSUM = O_BSTART + al((NA_MAX_BINS + 1) * sizeof(int));
constexpr size_t O_INTS = O_BTSUM + al(NA_TSUM * sizeof(int));      // 6 int arrays
constexpr size_t INT_ARR = al((size_t)NA_MAX_ATOMS * sizeof(int));
constexpr size_t O_OFFS = O_INTS + 6 * INT_ARR;                       // 4 double4 arrays
constexpr size_t OFF_ARR = al((size_t)NA_MAX_ATOMS * 4 * sizeof(double));
constexpr size_t O_PART = O_OFFS + 4 * OFF_ARR;
constexpr size_t SCRATCH_BYTES = O_PART + al((size_t)NA_TILES * NPART * sizeof(double));

// ~8.5 MB for 32,768 atoms
__device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

struct H1 {
    double h[9];
};

// Writes the launch descriptors into the scratch array (arguments arrive by
// value, so no host-to-device copy is needed) and clears the bin counts.
__global__ void k_noalloc_init(BandDev dv, BandParams bp, H1 cell, int ntiles) {
    unsigned char *base = g_noalloc_scratch;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0) {
        *(BandDev *)(base + O_BAND) = dv;
        *(BandParams *)(base + O_PARAMS) = bp;
        double *h1 = (double *)(base + O_H1);
        for (int k = 0; k < 9; ++k) h1[k] = cell.h[k];
        ImgRef r;
        r.band = 0;
        r.img = 0;
        *(ImgRef *)(base + O_IMG) = r;
    }
    Tile *tiles = (Tile *)(base + O_TILES);
    for (int t = tid; t < ntiles; t += gridDim.x * blockDim.x) {
        Tile tl;
        tl.band = 0;
        tl.img = 0;
        tl.t = t;
        tl.pad = 0;
        tiles[t] = tl;
    }
    int *cnt = (int *)(base + O_BCOUNT);
    for (int k = tid; k < NA_MAX_BINS; k += gridDim.x * blockDim.x) cnt[k] = 0;
}

// The device address of the array belongs to the CUDA context the module is
// loaded in (a cudaDeviceReset or a context of the caller's own makes a new
// one), so it is looked up once per context and cached under the context's
// process-unique id (cuCtxGetId; the driver functions are reached through
// the runtime's entry-point query, so no driver library is linked).
std::mutex g_mu;
std::map<unsigned long long, unsigned char *> g_base;
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;

// the array's device address in the current context, or nullptr
unsigned char *scratch_base() {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ctx_current || !g_ctx_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault,
                                             &q1) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) !=
                cudaSuccess ||
            q2 != cudaDriverEntryPointSuccess)
            return nullptr;
        g_ctx_current = (CtxGetCurrentFn)f1;
        g_ctx_id = (CtxGetIdFn)f2;
    }
    // make the runtime bind the device's context to this thread first
    if (cudaFree(nullptr) != cudaSuccess) return nullptr;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx || g_ctx_id(ctx, &id) != CUDA_SUCCESS)
        return nullptr;
    auto it = g_base.find(id);
    if (it != g_base.end()) return it->second;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return nullptr;
    g_base[id] = (unsigned char *)p;
    return (unsigned char *)p;
}

}  // namespace

extern "C" int cfneb_lj_evaluate_noalloc(const double *d_positions, int32_t n_atoms,
                                         const double *cell, double eps, double sigma,
                                         double rc, int32_t shift_energy, double *d_energy,
                                         double *d_forces, double *d_virial, void *cuda_stream) {
    if (!d_positions || !cell || n_atoms <= 0) return CFNEB_ERR_INVALID_ARG;
    if (n_atoms > NA_MAX_ATOMS) return CFNEB_ERR_INVALID_ARG;
    for (int k = 0; k < 9; ++k)
        if (!std::isfinite(cell[k])) return CFNEB_ERR_INVALID_ARG;
    if (!std::isfinite(eps) || !std::isfinite(sigma) || !std::isfinite(rc) || !(eps > 0) ||
        !(sigma > 0) || !(rc > 0))
        return CFNEB_ERR_INVALID_ARG;
    if (!(std::fabs(det3(cell)) > 0)) return CFNEB_ERR_INVALID_ARG;
    // the cell list reaches MAX_STENCIL bins to each side: every lattice
    // direction must be at least rc / MAX_STENCIL wide
    {
        const double vol = std::fabs(det3(cell));
        for (int a = 0; a < 3; ++a) {
            const double *u = cell + 3 * ((a + 1) % 3), *v = cell + 3 * ((a + 2) % 3);
            const double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2],
                         cz = u[0] * v[1] - u[1] * v[0];
            const double w = vol / std::sqrt(cx * cx + cy * cy + cz * cz);
            if (!(rc < MAX_STENCIL * w * 0.999)) return CFNEB_ERR_INVALID_ARG;
        }
    }
    // the device address of the array in the current context (host code
    // may not use the symbol itself as a pointer)
    unsigned char *base = scratch_base();
    if (!base) return CFNEB_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int n = n_atoms;
    BandDev dv;
    memset(&dv, 0, sizeof(dv));
    dv.n = n;
    dv.rows = n + 3;
    dv.ncap = NA_IMAGES;
    dv.nbins_cap = NA_MAX_BINS;
    dv.atpi = (n + TILE - 1) / TILE;
    dv.rtpi = (n + 3 + RTILE - 1) / RTILE;
    dv.X = base + O_X;
    dv.F = base + O_F;
    dv.Fneb = dv.F;  // not used by an evaluation
    dv.v = dv.F;
    dv.sc = (ImgScalars *)(base + O_SC);
    dv.bp = (BandParams *)(base + O_PARAMS);
    dv.bin_count = (int *)(base + O_BCOUNT);
    dv.bin_start = (int *)(base + O_BSTART);
    dv.bin_tsum = (int *)(base + O_BTSUM);
    dv.tsum_cap = NA_TSUM;
    dv.atom_bin = (int *)(base + O_INTS + 0 * INT_ARR);
    dv.atom_rank = (int *)(base + O_INTS + 1 * INT_ARR);
    dv.slot_unsorted = (int *)(base + O_INTS + 2 * INT_ARR);
    dv.slot_atom = (int *)(base + O_INTS + 3 * INT_ARR);
    dv.slot_bin = (int *)(base + O_INTS + 4 * INT_ARR);
    dv.atom_slot = (int *)(base + O_INTS + 5 * INT_ARR);
    dv.atom_off = base + O_OFFS + 0 * OFF_ARR;
    dv.slot_off = base + O_OFFS + 1 * OFF_ARR;
    dv.atom_off_lo = base + O_OFFS + 2 * OFF_ARR;
    dv.slot_off_lo = base + O_OFFS + 3 * OFF_ARR;
    dv.atom_part = (double *)(base + O_PART);

    BandParams bp;
    memset(&bp, 0, sizeof(bp));
    for (int k = 0; k < 9; ++k) bp.h0[k] = cell[k];
    inv3(bp.h0, bp.h0inv);
    bp.c = (double)n;
    bp.rc = rc;
    bp.bin_w = rc;
    bp.row_refine = 1;
    bp.ftol = -1.0;
    bp.move_limit = 0;
    bp.filter = 1;
    bp.variant = CFNEB_ROTFREE_B;
    bp.n = n;
    bp.N = NA_IMAGES;
    bp.kind = CFNEB_LJ;
    bp.ci = -1;
    const double sr6 = std::pow(sigma / rc, 6.0);
    bp.pot[0] = eps;
    bp.pot[1] = sigma;
    bp.pot[2] = rc;
    bp.pot[3] = shift_energy ? 4.0 * eps * (sr6 * sr6 - sr6) : 0.0;
    H1 h1;
    for (int k = 0; k < 9; ++k) h1.h[k] = cell[k];

    BandDev *d_band = (BandDev *)(base + O_BAND);
    const Tile *d_tiles = (const Tile *)(base + O_TILES);
    const ImgRef *d_img = (const ImgRef *)(base + O_IMG);
    const double *d_h1 = (const double *)(base + O_H1);
    k_noalloc_init<<<32, 256, 0, s>>>(dv, bp, h1, dv.atpi);
    launch_setup<double>(d_positions, d_positions, nullptr, n, NA_IMAGES, d_band, s, d_h1);
    launch_mapback<double>(d_img, 1, d_band, 1, s);  // forced: the scratch record is reused
    launch_bin_assign<double>(d_tiles, dv.atpi, d_band, s);
    launch_bin_scan(d_img, 1, NA_MAX_BINS, d_band, s, 0);
    launch_bin_scan(d_img, 1, NA_MAX_BINS, d_band, s, 1);
    launch_bin_scan(d_img, 1, NA_MAX_BINS, d_band, s, 2);
    launch_bin_scatter(d_tiles, dv.atpi, d_band, s);
    launch_bin_order<double>(d_img, 1, NA_MAX_BINS, d_band, s);
    launch_lj<double>(d_tiles, dv.atpi, d_band, s);
    launch_image_finalize<double>(d_img, 1, d_band, s);
    if (cudaGetLastError() != cudaSuccess) return CFNEB_ERR_CUDA;
    const ImgScalars *sc0 = (const ImgScalars *)(base + O_SC);
    if (d_energy &&
        cudaMemcpyAsync(d_energy, &sc0->E, sizeof(double), cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess)
        return CFNEB_ERR_CUDA;
    if (d_virial &&
        cudaMemcpyAsync(d_virial, sc0->V, 9 * sizeof(double), cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess)
        return CFNEB_ERR_CUDA;
    // image 0's atom rows of F: Cartesian forces (D = I for h0 = cell)
    if (d_forces && cudaMemcpyAsync(d_forces, base + O_F, (size_t)n * 3 * sizeof(double),
                                    cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return CFNEB_ERR_CUDA;
    // the status word the kernels raise, and the energy (a non-finite
    // energy marks overlapping atoms): read back once the work is done
    int bits = 0;
    double e = 0.0;
    const BandParams *d_bp = (const BandParams *)(base + O_PARAMS);
    if (cudaMemcpyAsync(&bits, &d_bp->status, sizeof(int), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(&e, &sc0->E, sizeof(double), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return CFNEB_ERR_CUDA;
    if (bits & ST_NONFINITE || !std::isfinite(e)) return CFNEB_ERR_NONFINITE;
    if (bits & ST_NOT_SPD) return CFNEB_ERR_NOT_SPD;
    if (bits & ST_NBR_OVERFLOW) return CFNEB_ERR_NBR_OVERFLOW;
    return CFNEB_OK;
}
