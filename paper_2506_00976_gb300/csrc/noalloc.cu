// noalloc.cu -- a lazy c-transform entry point that allocates no memory.
//
// Some callers cannot allocate device memory at the point where they need a
// c-transform: code that runs while a memory pool is frozen or exhausted,
// callers that own every byte of their device budget up front, and plugins
// loaded into a host process that forbids new allocations.  For them this
// entry point runs the same kernels as qwb_ctransform, but every scratch
// buffer lives in one statically sized device array that exists for the
// lifetime of the loaded library.
//
// Limits and sharing rules (also stated in include/qwb.h):
//   * N <= 256; larger grids are rejected;
//   * every call uses the same array, which keeps the previous call's
//     contents; each call rewrites everything it reads before reading it;
//   * calls whose GPU work overlaps (different streams, or host threads
//     racing) corrupt each other's results: serialise them;
//   * the first call on a device does the set-up: it looks up the array's
//     device address and, under lazy module loading (the CUDA default), loads
//     the kernels, which itself takes device memory.  Make that first call
//     while memory can still be allocated.
//
// The launch plan (pair descriptor and work items) is written into the array
// by a set-up kernel from values passed by value, so no call copies host
// memory to the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>   // per-device address table, filled once per device

#include "common.cuh"
#include "kernels.h"

namespace qwb {
namespace {

constexpr int kMaxN = 256;
constexpr int kMaxM = kMaxN * kMaxN;
constexpr int kMaxItems = 512;

// Scratch layout (bytes): FP32 copy of h, FP32 result accumulator, FP32 cost
// table, one pair descriptor, the work-item list.
constexpr size_t kOffH = 0;
constexpr size_t kOffOut = kOffH + sizeof(float) * kMaxM;
constexpr size_t kOffTab = kOffOut + sizeof(float) * kMaxM;
constexpr size_t kOffTabHi = kOffTab + sizeof(float) * kMaxM;
constexpr size_t kOffDesc = kOffTabHi + sizeof(float) * kMaxM;
constexpr size_t kOffItems = kOffDesc + ((sizeof(PairDev) + 255) / 256) * 256;
constexpr size_t kScratchBytes = kOffItems + sizeof(CtItem) * kMaxItems;

// 1 MiB + a few KiB, held by every GPU that loads the library until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct DeviceScratch {
    bool ready = false;
    unsigned char* ptr = nullptr;
};
std::mutex g_mtx;
std::vector<DeviceScratch> g_dev;

int scratch_for_current_device(unsigned char** out) {
    int dev = 0;
    QWB_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mtx);
    if ((int)g_dev.size() <= dev) g_dev.resize(dev + 1);
    if (!g_dev[dev].ready) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
        g_dev[dev].ptr = static_cast<unsigned char*>(p);
        g_dev[dev].ready = true;
    }
    *out = g_dev[dev].ptr;
    return QWB_OK;
}

// Writes the pair descriptor and the work items into the static scratch:
// tile t (CT_TILE outputs from t * CT_TILE), input-row split r (input rows
// [r * rows, min(N, (r + 1) * rows))), item index t * splits + r -- the same
// items the host plan of qwb_ctransform builds.
__global__ void noalloc_plan_kernel(PairDev P, PairDev* __restrict__ desc, CtItem* __restrict__ items,
                                    int rows, int splits, int n_items) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *desc = P;
    if (i < n_items) {
        const int t = i / splits, r = i - t * splits;
        const int r0 = r * rows;
        items[i] = CtItem{0, t * CT_TILE, r0, min(rows, P.N - r0)};
    }
}

}  // namespace
}  // namespace qwb

using namespace qwb;

extern "C" int qwb_ctransform_noalloc(int32_t N, double p, const double* h_d, double* out_d,
                                      void* stream) {
    if (!h_d || !out_d) {
        set_last_error("qwb_ctransform_noalloc: null pointer");
        return QWB_ERR_INVALID_ARG;
    }
    if (N < 1 || N > kMaxN) {
        set_last_error("qwb_ctransform_noalloc: N must be in [1, 256] (the static scratch holds 256 x 256 grids)");
        return QWB_ERR_UNSUPPORTED;
    }
    if (!(p >= 1.0)) {
        set_last_error("qwb_ctransform_noalloc: p must be >= 1");
        return QWB_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* base = nullptr;
    int st = scratch_for_current_device(&base);
    if (st) return st;
    float* h32 = reinterpret_cast<float*>(base + kOffH);
    float* out32 = reinterpret_cast<float*>(base + kOffOut);
    float* tab_lo = reinterpret_cast<float*>(base + kOffTab);
    float* tab_hi = reinterpret_cast<float*>(base + kOffTabHi);
    PairDev* desc = reinterpret_cast<PairDev*>(base + kOffDesc);
    CtItem* items = reinterpret_cast<CtItem*>(base + kOffItems);

    // launch plan: 4096-output tiles, each split into about two items per SM;
    // the staged input rows of an item must fit in shared memory
    int dev = 0, sm = 148;
    QWB_CUDA(cudaGetDevice(&dev));
    QWB_CUDA(cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev));
    const int m = N * N;
    const int tiles = (m + CT_TILE - 1) / CT_TILE;
    const int splits0 = std::max(1, std::min(std::min(N, kMaxItems / tiles), (2 * sm + tiles - 1) / tiles));
    const int rows_smem = (227 * 1024) / (int)(sizeof(float) * N);   // >= 227 for N <= 256
    const int rows = std::min((N + splits0 - 1) / splits0, rows_smem);
    const int splits = (N + rows - 1) / rows;                        // every split non-empty
    const int n_items = tiles * splits;                              // <= 512 (splits <= max(splits0, 2))
    if (n_items > kMaxItems) {
        set_last_error("qwb_ctransform_noalloc: launch plan exceeds the static item list");
        return QWB_ERR_UNSUPPORTED;
    }
    PairDev P;
    std::memset(&P, 0, sizeof(P));
    P.N = N; P.kappa = N; P.n = 1; P.M = 1; P.p = p;
    P.d = 2; P.m = N * N; P.rows = N;
    P.ctab_lo = tab_lo; P.ctab_hi = tab_hi;
    P.fhat = h32; P.g = out32;

    // everything the kernels read is rewritten here, so the previous call's
    // contents never leak into this one; the plan travels as kernel arguments
    noalloc_plan_kernel<<<(n_items + 255) / 256, 256, 0, s>>>(P, desc, items, rows, splits, n_items);
    QWB_LAUNCHED();
    if (p != 2.0 && (st = launch_cost_tables(N, p, false, tab_lo, tab_hi, s))) return st;
    if ((st = launch_to_work(h_d, h32, out32, m, false, s))) return st;   // h rounded up, out = +inf
    CtConfig cfg;
    cfg.R = ct_pick_r(N, 8);
    cfg.TC = cfg.R;
    cfg.threads = 256;
    cfg.in_rows = rows;
    cfg.p2 = (p == 2.0);
    if ((st = launch_ctransform(desc, items, n_items, 0, cfg, N, false, 0, s))) return st;
    return launch_from_work(out32, out_d, m, false, s);
}
