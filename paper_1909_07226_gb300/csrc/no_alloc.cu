// Gridding without any device allocation: idg_grid_no_alloc.
//
// idg_grid takes its subgrid scratch from a stream-ordered memory pool.  Some
// callers cannot allocate device memory at the time they grid: a real-time
// pipeline that reserves its whole memory budget up front, or a host framework
// whose own allocator already owns all free device memory.  For them a new
// allocation may fail in the middle of a run or implicitly synchronise the
// device.  This variant runs the same gridder, subgrid FFT and adder kernels,
// but keeps the subgrid scratch in a fixed array compiled into the library.
//
// The array is a file-scope __device__ variable of kStaticScratchBytes.  Every
// GPU on which the library's module is loaded holds it until the process
// exits.  Host code cannot use the array's name as a device address, so its
// address is looked up once per device with cudaGetSymbolAddress, with that
// device current, and cached.  With CUDA's lazy module loading that first
// lookup is also what loads this module, and with it the 64 MiB array, on the
// device: the first call on each device may therefore fail for lack of memory
// or synchronise the device, and belongs before the caller reserves its memory
// and before any stream capture.  A call with a plan of no subgrids does only
// this lookup, so it serves as the warm-up.  The cached address assumes the
// device's context lives as long as the process: after cudaDeviceReset the
// cached address is stale, and the call is not supported.
//
// The compensated adder needs a grid-sized compensation buffer, which this call
// cannot allocate, so plans with IDG_ADDER_COMPENSATED are refused.  The sorted
// adder (IDG_ADDER_SORTED) needs no buffer: its plans run in plan order.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "idg_internal.h"

static constexpr size_t kStaticScratchBytes = size_t(64) << 20;   // 64 MiB

// The scratch itself: one per device that loads this module, alive until exit.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace idg {
namespace {

std::mutex g_addr_mu;
void *g_addr[64] = {};

// Device address of g_static_scratch on `device` (which must be current).
idg_status static_scratch_address(int device, void **out) {
    if (device < 0 || device >= 64) return fail(IDG_ERR_INVALID_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
        g_addr[device] = p;
    }
    *out = g_addr[device];
    return IDG_OK;
}

}  // namespace
}  // namespace idg

using namespace idg;

extern "C" idg_status idg_grid_no_alloc(const idg_plan *p, const void *vis, const uint8_t *flags,
                                        const void *aterms, const float *taper, void *grid, idg_stream stream) {
    if (!p) return fail(IDG_ERR_INVALID_ARG, "plan is NULL");
    if (!vis) return fail(IDG_ERR_INVALID_ARG, "d_vis is NULL");
    if (!grid) return fail(IDG_ERR_INVALID_ARG, "d_grid is NULL");
    if (!(taper = p->taper_or_default(taper)) && p->device >= 0)
        return fail(IDG_ERR_INVALID_ARG, "the taper is NULL and the plan has no default taper");
    if (p->opts.adder_mode == IDG_ADDER_COMPENSATED)
        return fail(IDG_ERR_UNSUPPORTED,
                    "idg_grid_no_alloc: the compensated adder needs a grid-sized buffer that this call cannot "
                    "allocate; use a plan with IDG_ADDER_ATOMIC or idg_grid");
    if (!gridder_supported(p->L))
        return fail(IDG_ERR_UNSUPPORTED, "subgrid size " + std::to_string(p->L) + " is not compiled in");
    if (p->device < 0) return fail(IDG_ERR_INVALID_ARG, "the plan was created without a CUDA device");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != p->device)
        return fail(IDG_ERR_INVALID_ARG, "plan was created on device " + std::to_string(p->device) +
                                             " but the current device is " + std::to_string(dev));
    const int64_t n = p->stats.n_subgrids;
    const size_t per = (size_t)p->L * p->L * 32;
    const size_t need = (size_t)n * per;
    if (need > kStaticScratchBytes)
        return fail(IDG_ERR_INVALID_ARG,
                    "idg_grid_no_alloc: the plan's " + std::to_string(n) + " subgrids of " + std::to_string(p->L) +
                        "x" + std::to_string(p->L) + " need " + std::to_string(need) +
                        " bytes of scratch; the built-in scratch holds " + std::to_string(kStaticScratchBytes) +
                        " bytes (" + std::to_string(kStaticScratchBytes / per) + " subgrids of this size)");
    void *scratch = nullptr;
    idg_status st = static_scratch_address(dev, &scratch);
    if (st != IDG_OK || n == 0) return st;
    // The gridder writes every pixel of every subgrid slot it uses before the
    // FFT and the adder read it, so nothing in the scratch has to start at zero.
    cudaStream_t s = (cudaStream_t)stream;
    const Geometry g = p->geometry();
    // (the sorted adder takes the subgrids in plan order: slot i holds plan index i)
    const bool sorted = p->opts.adder_mode == IDG_ADDER_SORTED;
    const SubgridSet all = sorted ? SubgridSet{nullptr, 0, n, p->kp_plan.data()}
                                  : SubgridSet{p->d_order, 0, n, p->kp_order.data()};
    st = launch_gridder(g, all, p->kernel_variant(IDG_KERNEL_GRIDDER), vis, flags, aterms, taper, scratch, s);
    if (st == IDG_OK) st = launch_subgrid_fft(p, n, -1, scratch, s);
    if (st == IDG_OK)
        st = sorted ? launch_adder_sorted(g, all, scratch, grid,
                                          SortedTiles{p->d_tile_ids, p->d_tile_first, p->d_tile_sub, p->n_tiles_sorted,
                                                      p->n_heavy_sorted}, s)
                    : launch_adder(g, all, scratch, grid, s);
    return st;
}
