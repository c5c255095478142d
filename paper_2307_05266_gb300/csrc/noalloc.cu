// Allocation-free permeability reduction.
//
// Callers that run inside a memory pool they do not own, inside an already-captured CUDA
// graph, or under a framework that forbids device allocation after start-up cannot let
// this library call cudaMalloc.  schur_permeability_noalloc serves them: it sums a
// caller-owned velocity field over the unknown faces with the same block-partial
// reduction as the solver, and keeps its scratch (the block partials and the block
// ticket) in a file-scope static device array instead of allocated memory.
//
// The array is reserved in every device context that loads this library and stays there
// until the process exits.  All calls on a device share it, so calls that overlap on the
// GPU (two streams, or two host threads) race on it and must be serialised by the caller.
#include <mutex>

#include "../../include/schur.h"
#include "internal.h"

namespace schur {
namespace {

constexpr int kStaticBlocks = 4096;                 // one block per chunk of faces
constexpr long long kStaticChunk = 2048;            // faces per block
constexpr long long kStaticMaxFaces = kStaticBlocks * kStaticChunk;  // 8,388,608

struct StaticScratch {
    double partials[kStaticBlocks * 3];  // per-block sums of u_x, u_y, u_z
    unsigned int ticket;                 // blocks finished; must start at 0
};

static __device__ __align__(256) StaticScratch g_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
// Per device: the array's device address and the id of the context it was looked up in.
// A device reset (cudaDeviceReset, which some host frameworks call) replaces the primary
// context and reloads the module, so the address is looked up again when the current
// context's id differs from the cached one.
StaticScratch* g_scratch_ptr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

// Driver entry points for the context id, resolved through the runtime (the library does
// not link the driver library directly).
typedef int (*CtxGetCurrentFn)(void** ctx);
typedef int (*CtxGetIdFn)(void* ctx, unsigned long long* id);

cudaError_t current_context_id(unsigned long long* id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000,
                                                         cudaEnableDefault, &q1);
        if (e != cudaSuccess) return e;
        e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess) return e;
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return cudaErrorNotSupported;
        get_current = (CtxGetCurrentFn)f1;
        get_id = (CtxGetIdFn)f2;
    }
    void* ctx = nullptr;
    if (get_current(&ctx) != 0 || !ctx) return cudaErrorDeviceUninitialized;
    return get_id(ctx, id) == 0 ? cudaSuccess : cudaErrorUnknown;
}

__global__ void k_perm_static(const double* __restrict__ u, const uint8_t* __restrict__ flags,
                              long long stride, int d, long long ncell,
                              StaticScratch* sc, double* __restrict__ k_out) {
    double v[3] = {0.0, 0.0, 0.0};
    const long long n = (long long)d * stride;
    const long long b0 = (long long)blockIdx.x * kStaticChunk;
    for (long long i = b0 + threadIdx.x; i < b0 + kStaticChunk && i < n; i += blockDim.x) {
        const int a = (int)(i / stride);
        const double ui = (flags[i] & 1) ? u[i] : 0.0;
        v[0] += (a == 0) ? ui : 0.0;
        v[1] += (a == 1) ? ui : 0.0;
        v[2] += (a == 2) ? ui : 0.0;
    }
    if (reduce_last_block<3>(v, sc->partials, &sc->ticket) && threadIdx.x == 0) {
        for (int a = 0; a < 3; ++a) k_out[a] = a < d ? v[a] / (double)ncell : 0.0;
    }
}

}  // namespace
}  // namespace schur

using namespace schur;

extern "C" int schur_permeability_noalloc(const double* u, const uint8_t* flags, int ndim,
                                          const int64_t dims[3], int64_t face_stride,
                                          void* stream, double* k_dev) {
    if (!u || !flags || !dims || !k_dev)
        return schur_set_error_internal(SCHUR_EINVAL, "null argument");
    if (ndim != 2 && ndim != 3) return schur_set_error_internal(SCHUR_EINVAL, "ndim must be 2 or 3");
    const long long nz = ndim == 3 ? dims[2] : 1;
    if (dims[0] < 2 || dims[1] < 2 || nz < 1 || (ndim == 3 && nz < 2))
        return schur_set_error_internal(SCHUR_EINVAL, "every extent must be >= 2");
    const long long ncell = dims[0] * dims[1] * nz;
    if (face_stride < ncell)
        return schur_set_error_internal(SCHUR_EINVAL, "face_stride must be >= the cell count");
    const long long n = (long long)ndim * face_stride;
    if (n > kStaticMaxFaces)
        return schur_set_error_internal(
            SCHUR_EINVAL, "ndim * face_stride exceeds the static scratch limit of 8388608 faces");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return schur_set_error_internal(SCHUR_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return schur_set_error_internal(SCHUR_EINVAL, "device ordinal beyond 63");
    StaticScratch* sc = nullptr;
    {
        // set-up, once per device (and again after a device reset), with that device
        // current: the host-side name of the static array is not a device address, so ask
        // the runtime for the real one
        std::lock_guard<std::mutex> lock(g_mutex);
        unsigned long long ctx = 0;
        e = current_context_id(&ctx);
        if (e == cudaErrorDeviceUninitialized) {
            // no context on this thread yet: the symbol lookup below creates the primary
            // context, after which its id can be read
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_scratch);
            if (e == cudaSuccess) e = current_context_id(&ctx);
        }
        if (e != cudaSuccess) return schur_set_error_internal(SCHUR_ECUDA, cudaGetErrorString(e));
        if (!g_scratch_ptr[dev] || g_scratch_ctx[dev] != ctx) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess)
                return schur_set_error_internal(SCHUR_ECUDA, cudaGetErrorString(e));
            g_scratch_ptr[dev] = (StaticScratch*)p;
            g_scratch_ctx[dev] = ctx;
        }
        sc = g_scratch_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    // the ticket must start at zero; the partials are fully rewritten by every call
    e = cudaMemsetAsync(&sc->ticket, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return schur_set_error_internal(SCHUR_ECUDA, cudaGetErrorString(e));
    const unsigned blocks = (unsigned)((n + kStaticChunk - 1) / kStaticChunk);
    k_perm_static<<<blocks, 256, 0, s>>>(u, flags, face_stride, ndim, ncell, sc, k_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return schur_set_error_internal(SCHUR_ECUDA, cudaGetErrorString(e));
    return SCHUR_OK;
}
