// Device helpers shared by the Krylov translation units (krylov.cu: Jacobi-preconditioned
// inner CG, outer Schur CG, mixed precision; mg.cu: multigrid-preconditioned inner CG):
// loop macros, the Krylov scalar updates, the compact layout and its stencil phases,
// block and grid sums of the persistent kernels, and the host-side launch shapes.
#pragma once

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>

#include "internal.h"

namespace schur {

#define TILE_LOOP_BEGIN(g)                                                        \
    const int gx_ = ((g).nx + kTileX - 1) / kTileX;                               \
    const int gy_ = ((g).ny + kTileY - 1) / kTileY;                               \
    const long long nt_ = (long long)gx_ * gy_ * (g).nz;                          \
    for (long long t_ = blockIdx.x; t_ < nt_; t_ += gridDim.x) {                  \
        const int x = (int)(t_ % gx_) * kTileX + (int)threadIdx.x;                \
        const int y = (int)((t_ / gx_) % gy_) * kTileY + (int)threadIdx.y;        \
        const int z = (int)(t_ / ((long long)gx_ * gy_));                         \
        if (x < (g).nx && y < (g).ny) {                                           \
            const long long c = ((long long)z * (g).ny + y) * (g).nx + x;
#define TILE_LOOP_END \
        }             \
    }

#define STREAM_LOOP(i, n) \
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (n); \
         i += (long long)gridDim.x * blockDim.x)

__device__ __forceinline__ bool is_thread0() { return threadIdx.x == 0 && threadIdx.y == 0; }

// per-type views of the ghost-count tables
template <typename T> struct Tab;
template <> struct Tab<double> {
    static __device__ __forceinline__ double diag(const Dev& g, int k) { return tab5(g.diag, k); }
    static __device__ __forceinline__ double w(const Dev& g, int k) { return tab5(g.wdiag, k); }
};
template <> struct Tab<float> {
    static __device__ __forceinline__ float diag(const Dev& g, int k) { return tab5f(g.diagf, k); }
    static __device__ __forceinline__ float w(const Dev& g, int k) { return tab5f(g.wdiagf, k); }
};

__device__ __forceinline__ void note_inner_status(Ctl* ctl, int st) {
    if (ctl && st > ctl->inner_status) ctl->inner_status = st;
}

// Finish an inner CG iteration (last block): returns the new loop condition.
__device__ __forceinline__ unsigned finish_inner(Ctl* ctl, CgState* st, double rz, double zz) {
    st->iter += 1;
    st->total += 1;
    st->first = 0;
    if (st->status == ST_BREAKDOWN) { note_inner_status(ctl, ST_BREAKDOWN); return 0u; }
    const double rel = sqrt(zz / st->zz0);
    st->rel = rel;
    if (rel < st->tol) { st->status = ST_OK; return 0u; }
    if (!(rel == rel)) { st->status = ST_BREAKDOWN; note_inner_status(ctl, ST_BREAKDOWN); return 0u; }
    if (st->iter >= st->max_iter) { st->status = ST_NOTCONV; note_inner_status(ctl, ST_NOTCONV); return 0u; }
    st->beta = rz / st->rho;
    st->rho = rz;
    return 1u;
}

__device__ __forceinline__ unsigned start_inner(Ctl* ctl, CgState* st, double rz, double zz) {
    st->iter = 0;
    st->first = 1;
    st->alpha = 0.0;
    st->beta = 0.0;
    st->rho = rz;
    st->zz0 = zz;
    if (zz == 0.0) { st->status = ST_OK; st->rel = 0.0; return 0u; }
    if (!(zz == zz) || isinf(zz)) {
        st->status = ST_BREAKDOWN;
        note_inner_status(ctl, ST_BREAKDOWN);
        return 0u;
    }
    st->status = ST_NOTCONV;
    st->rel = 1.0;
    return 1u;
}

// alpha = rho / p.q; returns false (breakdown) when p.q is not positive and finite.
__device__ __forceinline__ bool matvec_alpha(CgState* st, double dq) {
    if (!(dq > 0.0) || isinf(dq)) {
        st->status = ST_BREAKDOWN;
        st->alpha = 0.0;
        return false;
    }
    st->alpha = st->rho / dq;
    return true;
}

__device__ __forceinline__ void finish_matvec(Ctl* ctl, CgState* st, double dq, int slot) {
    if (!matvec_alpha(st, dq)) set_cond(ctl, slot, 0u);
}

// ------------------------------------------------------------------------------------
// access patterns and the compact layout
// ------------------------------------------------------------------------------------
// Streaming kernels: a warp owns U chunks of 32 consecutive compact entries per step
// (lane l takes entry base + l + 32 j), every load is a coalesced row, and each thread
// has U independent loads in flight (4 in FP32; 2 in FP64, whose kernels are bound by
// the FP64 pipe and gain more from resident warps than from deeper unrolling).
template <typename T> struct StreamU { static constexpr int v = 4; };
template <> struct StreamU<double> { static constexpr int v = 2; };

// 32-bit indices: entry counts stay below 2^31 (checked when a geometry is created).
#define WARP_STREAM_BEGIN_U(n, U)                                                         \
    {                                                                                     \
        const uint32_t n_ = (uint32_t)(n);                                                \
        const uint32_t lane_ = threadIdx.x & 31u;                                         \
        const uint32_t step_ = ((gridDim.x * blockDim.x) >> 5) * (32u * (U));             \
        for (uint32_t base_ = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (32u * (U)); \
             base_ < n_; base_ += step_) {                                                \
            uint32_t idx[U];                                                              \
            _Pragma("unroll") for (int j = 0; j < (U); ++j) idx[j] = base_ + lane_ + 32u * j;
#define WARP_STREAM_END \
        }               \
    }

// Hint: fetch the 128-byte line that holds *p into L2.  No register receives data and
// nothing waits on it, so a stream phase can ask for the entries of a later grid-stride
// step while its own loads are in flight.  Callers pass in-bounds addresses only.
__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Row bitmaps of the compact layout.
struct Compact {
    const uint32_t* ulist;   // [n_u] face index of unknown k
    const uint32_t* flist;   // [n_p] cell index of fluid cell m
    const uint8_t* ufl;      // [n_u] flag byte of unknown k
    const uint32_t* fmask;   // face rows (a, z, y): [d * nz * ny][W]
    const uint32_t* fbase;
    const uint32_t* cmask;   // cell rows (z, y): [nz * ny][W]
    const uint32_t* cbase;
    int W;
    long long n_u, n_p;
    const uint32_t* nbA;     // [2d][ldA] stencil neighbours of the unknown faces
    const uint32_t* nbS;     // [2d][ldS] neighbours of the fluid cells across open faces
    const uint32_t* codeS;   // [n_p] per direction 3 bits: 0 closed, 1 + ghost count
    long long ldA, ldS;
};

__device__ __forceinline__ bool wrap3(const Dev& g, int& x, int& y, int& z) {
    if (x < 0) { if (!g.per[0]) return false; x += g.nx; } else if (x >= g.nx) { if (!g.per[0]) return false; x -= g.nx; }
    if (y < 0) { if (!g.per[1]) return false; y += g.ny; } else if (y >= g.ny) { if (!g.per[1]) return false; y -= g.ny; }
    if (z < 0) { if (!g.per[2]) return false; z += g.nz; } else if (z >= g.nz) { if (!g.per[2]) return false; z -= g.nz; }
    return true;
}

// Compact index of the entry at position x of a row, or -1 when the bit is clear.
__device__ __forceinline__ long long row_rank(const uint32_t* __restrict__ mask,
                                              const uint32_t* __restrict__ base, long long row,
                                              int W, int x) {
    const long long wi = row * W + (x >> 5);
    const uint32_t m = mask[wi];
    const uint32_t bit = 1u << (x & 31);
    if (!(m & bit)) return -1;
    return (long long)base[wi] + __popc(m & (bit - 1u));
}

// Compact index of face (a, x, y, z) (wrapped; -1 outside a closed box or not unknown).
__device__ __forceinline__ long long face_rank(const Dev& g, const Compact& C, int a, int x,
                                               int y, int z) {
    if (!wrap3(g, x, y, z)) return -1;
    return row_rank(C.fmask, C.fbase, ((long long)a * g.nz + z) * g.ny + y, C.W, x);
}

// Compact index of fluid cell (x, y, z) (wrapped; -1 outside or solid).
__device__ __forceinline__ long long cell_rank(const Dev& g, const Compact& C, int x, int y, int z) {
    if (!wrap3(g, x, y, z)) return -1;
    return row_rank(C.cmask, C.cbase, (long long)z * g.ny + y, C.W, x);
}

// Value of a compact face vector at face (a, x, y, z), 0 when the face is not an unknown.
template <typename T>
__device__ __forceinline__ double face_valc(const Dev& g, const Compact& C, const T* __restrict__ u,
                                            int a, int x, int y, int z) {
    const long long k = face_rank(g, C, a, x, y, z);
    return k < 0 ? 0.0 : (double)u[k];
}

// Decode a face index of [d][stride] (or a cell index) into component and coordinates.
struct FaceAt {
    int a, x, y, z;
    long long c;
};
__device__ __forceinline__ FaceAt decode_face(const Dev& g, uint32_t i) {
    FaceAt r;
    const uint32_t s = (uint32_t)g.stride;
    r.a = (i >= s) + (i >= 2u * s);
    const uint32_t c = i - (uint32_t)r.a * s;
    const uint32_t plane = (uint32_t)g.nx * (uint32_t)g.ny;
    r.z = (int)(c / plane);
    const uint32_t rem = c - (uint32_t)r.z * plane;
    r.y = (int)(rem / (uint32_t)g.nx);
    r.x = (int)(rem - (uint32_t)r.y * (uint32_t)g.nx);
    r.c = c;
    return r;
}

// Entries per thread and step of the stencil phases (independent gathers in flight).
template <typename T> struct MvU { static constexpr int v = 4; };
template <> struct MvU<double> { static constexpr int v = 2; };
// ... and in the persistent loop kernel, where register pressure sets the occupancy.
template <typename T> struct LoopMvU { static constexpr int v = 2; };

// Per-block copies of the ghost-count tables in shared memory: a lookup is one indexed
// shared load (no select chain, and nothing for the compiler to keep in registers across
// the phases of the loop kernel).  w[0] = 0 is the weight of a closed face, w[1 + g] the
// Jacobi weight 1 / (2d + g), diag[g] = 2d + g.
template <typename T>
struct Tabs {
    T diag[5];
    T w[6];
};

template <typename T>
__device__ __forceinline__ void load_tabs(const Dev& g, Tabs<T>& t) {
    const int i = threadIdx.x;
    if (i < 5) {
        t.diag[i] = Tab<T>::diag(g, i);
        t.w[i + 1] = Tab<T>::w(g, i);
    }
    if (i == 5) t.w[0] = (T)0;
    __syncthreads();
}

// q = A' p; returns this thread's part of p.q.  The neighbour indices come from the table
// (coalesced rows); missing neighbours point at the zero entry p[n_u].
template <typename T, int U = MvU<T>::v>
__device__ __forceinline__ T phaseA_matvec(const Tabs<T>& t, const Dev& g, const Compact& C,
                                           const T* __restrict__ pv, T* __restrict__ qv) {
    T acc = (T)0;
    const uint32_t n = (uint32_t)C.n_u;
    const int ne = 2 * g.d;
    WARP_STREAM_BEGIN_U(n, U)
        uint32_t nb[U][6];
        int gh[U];
        T pc[U];
#pragma unroll
        for (int j = 0; j < U; ++j)
            if (idx[j] < n) {
#pragma unroll
                for (int e = 0; e < 6; ++e)
                    nb[j][e] = e < ne ? __ldcs(C.nbA + e * C.ldA + idx[j]) : n;
                gh[j] = C.ufl[idx[j]] >> 1;
                pc[j] = pv[idx[j]];
            }
#pragma unroll
        for (int j = 0; j < U; ++j)
            if (idx[j] < n) {
                T sv[6];
#pragma unroll
                for (int e = 0; e < 6; ++e) sv[e] = pv[nb[j][e]];
                const T s = ((sv[0] + sv[1]) + (sv[2] + sv[3])) + (sv[4] + sv[5]);
                const T out = t.diag[gh[j]] * pc[j] - s;
                qv[idx[j]] = out;
                acc += pc[j] * out;
            }
    WARP_STREAM_END
    return acc;
}

// q = S-hat p; returns this thread's part of p.q.  FP64 (bound by the FP64 pipe) forms
// diag(S-hat) p_c minus the weighted neighbour sum; FP32 sums the weighted differences
// (p_c - p_nb), which vanish exactly on constants.  Closed faces point at the zero entry
// p[n_p] with weight 0.
template <typename T, int U = MvU<T>::v>
__device__ __forceinline__ T phaseS_matvec(const Tabs<T>& t, const Dev& g, const Compact& C,
                                           const T* __restrict__ dS, const T* __restrict__ pv,
                                           T* __restrict__ qv) {
    T acc = (T)0;
    const uint32_t n = (uint32_t)C.n_p;
    const int ne = 2 * g.d;
    WARP_STREAM_BEGIN_U(n, U)
        uint32_t nb[U][6], code[U];
        T pc[U], dg[U];
#pragma unroll
        for (int j = 0; j < U; ++j)
            if (idx[j] < n) {
#pragma unroll
                for (int e = 0; e < 6; ++e)
                    nb[j][e] = e < ne ? __ldcs(C.nbS + e * C.ldS + idx[j]) : n;
                code[j] = __ldcs(C.codeS + idx[j]);
                pc[j] = pv[idx[j]];
                if constexpr (sizeof(T) == 8) dg[j] = dS[idx[j]];
            }
#pragma unroll
        for (int j = 0; j < U; ++j)
            if (idx[j] < n) {
                T sv[6];
#pragma unroll
                for (int e = 0; e < 6; ++e) sv[e] = pv[nb[j][e]];
                T out;
                if constexpr (sizeof(T) == 8) {
                    T s = t.w[code[j] & 7u] * sv[0];
#pragma unroll
                    for (int e = 1; e < 6; ++e) s += t.w[(code[j] >> (3 * e)) & 7u] * sv[e];
                    out = dg[j] * pc[j] - s;
                } else {
                    out = (T)0;
#pragma unroll
                    for (int e = 0; e < 6; ++e)
                        out += t.w[(code[j] >> (3 * e)) & 7u] * (pc[j] - sv[e]);
                }
                qv[idx[j]] = out;
                acc += pc[j] * out;
            }
    WARP_STREAM_END
    return acc;
}

// Block sum of K doubles, result in every thread (one warp adds through shared memory).
template <int K, int NT = kBlock>
__device__ __forceinline__ void block_sum(double (&v)[K]) {
    __shared__ double sm[K][NT];
    __shared__ double out[K];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nthr = blockDim.x;
#pragma unroll
    for (int k = 0; k < K; ++k) sm[k][tid] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double x = 0.0;
            for (int j = lane; j < nthr; j += 32) x += sm[k][j];
            x = warp_sum(x);
            if (lane == 0) out[k] = x;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = out[k];
    __syncthreads();
}

// Grid sum of K doubles, identical in every block: block sums go to part[block][K], all
// blocks meet at a barrier, then warp 0 of each block adds the gridDim.x partials in a
// fixed order (lane l the partials l, l + 32, ..., then a shuffle tree) and shares the
// totals through shared memory.  Returns false when the barrier failed.
template <int K, int NT = kBlock>
__device__ __forceinline__ bool grid_sum(double (&v)[K], double* part, Ctl* ctl, unsigned& target) {
    __shared__ double tot[K];
    block_sum<K, NT>(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) part[(size_t)blockIdx.x * K + k] = v[k];
    }
    if (!grid_barrier(ctl, target)) return false;
    if (threadIdx.x < 32) {
        double acc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = 0.0;
        for (unsigned i = threadIdx.x; i < gridDim.x; i += 32) {
#pragma unroll
            for (int k = 0; k < K; ++k) acc[k] += __ldcg(&part[(size_t)i * K + k]);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            acc[k] = warp_sum(acc[k]);
            if (threadIdx.x == 0) tot[k] = acc[k];
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = tot[k];
    return true;
}

// Hides a value from the optimiser for one loop iteration, so that addresses derived
// from it are recomputed in each phase rather than kept live across the other phases of
// the loop kernel (the loop kernel is held to 85 registers by its launch bounds).
template <class P>
__device__ __forceinline__ P* opaque(P* p) {
    asm volatile("" : "+l"(p));
    return p;
}
__device__ __forceinline__ uint32_t opaque_u32(uint32_t v) {
    asm volatile("" : "+r"(v));
    return v;
}

static inline dim3 tblock() { return dim3(kTileX, kTileY, 1); }
static inline dim3 tgrid(const Handle& H) {
    const long long gx = (H.g.nx + kTileX - 1) / kTileX, gy = (H.g.ny + kTileY - 1) / kTileY;
    const long long nt = gx * gy * H.g.nz;
    return dim3((unsigned)(nt < H.target_blocks ? nt : H.target_blocks));
}
// Resident blocks of kBlock threads per SM for kernel k (cached per device and kernel).
static int resident_blocks(const void* k, size_t smem = 0, int threads = kBlock) {
    static std::mutex mu;
    static std::map<std::pair<std::pair<int, const void*>, std::pair<size_t, int>>, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_pair(std::make_pair(dev, k), std::make_pair(smem, threads));
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads, smem) != cudaSuccess || nb < 1) {
        (void)cudaGetLastError();
        nb = 1;
    }
    cache[key] = nb;
    return nb;
}

// Streaming grids: one block per kBlock x min_per_thread entries, at most one wave of
// resident blocks (nsm x min(blocks per SM of the launch shape, resident blocks of the
// kernel)), so that the grid-stride loops end together instead of leaving a partial last
// wave (and the cooperative loop kernels always fit).
template <class K>
static inline dim3 sgrid(const Handle& H, long long n, K k) {
    const long long per_block = (long long)kBlock * std::max(1, H.min_per_thread);
    const long long nb = (n + per_block - 1) / per_block;
    const long long cap = std::min<long long>(H.target_blocks,
                                              (long long)H.nsm * resident_blocks((const void*)k));
    return dim3((unsigned)std::max<long long>(1, std::min(nb, cap)));
}
static inline dim3 sblock() { return dim3(kBlock); }

// Grids of the persistent loop kernels.  In the single-solve shape (one entry per thread
// at least) a loop grid gives every thread kLoopMinPerThread entries but keeps one block
// per SM when the problem has that many rows: mid-size inner solves run faster on fewer,
// fuller blocks (cheaper barriers), small ones need the SMs for latency.  Shapes made for
// sharing the GPU keep their own entries per thread.
constexpr int kLoopMinPerThread = 4;
template <class K>
static inline dim3 lgrid(const Handle& H, long long n, K k, size_t smem = 0) {
    const long long cap = std::min<long long>(H.target_blocks,
                                              (long long)H.nsm * resident_blocks((const void*)k, smem));
    const long long rows = (n + kBlock - 1) / kBlock;
    long long nb;
    if (H.min_per_thread > 1) {
        const long long per_block = (long long)kBlock * H.min_per_thread;
        nb = (n + per_block - 1) / per_block;
    } else {
        const long long per_block = (long long)kBlock * kLoopMinPerThread;
        nb = std::max((n + per_block - 1) / per_block, std::min<long long>(H.nsm, rows));
    }
    return dim3((unsigned)std::max<long long>(1, std::min(nb, cap)));
}

static Compact compact_of(const Handle& H) {
    Compact C;
    C.ulist = H.ulist;
    C.flist = H.flist;
    C.ufl = H.ufl;
    C.fmask = H.fmask;
    C.fbase = H.fbase;
    C.cmask = H.cmask;
    C.cbase = H.cbase;
    C.W = H.W;
    C.n_u = H.n_u;
    C.n_p = H.n_p;
    C.nbA = H.nbA;
    C.nbS = H.nbS;
    C.codeS = H.codeS;
    C.ldA = H.ldA;
    C.ldS = H.ldS;
    return C;
}

// Buffers of one inner solve.
template <typename T>
struct InnerA {
    T *x, *r, *p, *q;
};
template <typename T>
struct InnerS {
    T *x, *r, *p, *q;
    const T* invd;
    const T* diag;   // diagonal of S-hat (read by the FP64 matvec only)
};
static InnerA<double> innerA64(Handle& H) { return {H.ax, H.ar, H.ap, H.aq}; }
static InnerA<float> innerA32(Handle& H) { return {H.axf, H.arf, H.apf, H.aqf}; }
static InnerS<double> innerS64(Handle& H) { return {H.sx, H.sr, H.sp, H.sq, H.invdSc, H.dSc}; }
static InnerS<float> innerS32(Handle& H) { return {H.sxf, H.srf, H.spf, H.sqf, H.invdSf, nullptr}; }

}  // namespace schur
