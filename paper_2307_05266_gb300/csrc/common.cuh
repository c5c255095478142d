// Shared device/host definitions of the GB300 Schur-complement Stokes solver.
//
// Layout in HBM (all buffers owned by one geometry handle):
//   mask   uint8  [n_cells]            C order [z][y][x], 1 = fluid
//   flags  uint8  [d][stride]          face (a, c) = lower face of cell c along axis a;
//                                      bit 0 unknown, bits 1..3 ghost (solid-solid) count
//   face vectors  T [d][stride]        0 on faces that are not unknowns
//   cell vectors  T [n_cells]          0 on solid cells
// stride = n_cells rounded up to 64 elements, so every component starts 512-byte aligned.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <string>
#include <vector>

namespace schur {

constexpr int kTileX = 32;             // threads along x in stencil tiles (one warp row)
constexpr int kTileY = 8;              // rows of a stencil tile
constexpr int kBlock = kTileX * kTileY;
constexpr int kMaxRed = 4;             // doubles reduced by one kernel at most
constexpr int kMaxBlocks = 4096;       // grid cap of every reducing kernel
constexpr int kSlots = 256;            // loop-condition slots per handle
constexpr double kZeroRhsRtol = 1e-12; // g == 0 when ||g|| <= this * || |B| |u| ||
constexpr int kMaxBig = 8;             // fluid components reduced by the full grid
constexpr long long kBigMin = 2048;    // smallest component treated as "big"

enum Status : int { ST_OK = 0, ST_NOTCONV = 3, ST_BREAKDOWN = 4, ST_BARRIER = 5 };

struct Dev {
    int nx, ny, nz, d;
    int per[3];
    long long ncell;
    long long stride;
    double h, hinv, h2inv, h2;
    // tables indexed by the ghost count g = 0..4 of a face (GB300 has little FP64
    // throughput, so no FP64 division or conversion appears in the hot loops)
    double diag[5];   // 2d + g: diagonal of the dimensionless operator h^2 A
    double wdiag[5];  // 1 / (2d + g)
    float diagf[5];   // the same in FP32
    float wdiagf[5];
};

__device__ __forceinline__ float tab5f(const float (&t)[5], int k) {
    float v = t[0];
    v = (k == 1) ? t[1] : v;
    v = (k == 2) ? t[2] : v;
    v = (k == 3) ? t[3] : v;
    v = (k == 4) ? t[4] : v;
    return v;
}

__device__ __forceinline__ double tab5(const double (&t)[5], int k) {
    double v = t[0];
    v = (k == 1) ? t[1] : v;
    v = (k == 2) ? t[2] : v;
    v = (k == 3) ? t[3] : v;
    v = (k == 4) ? t[4] : v;
    return v;
}

// One Krylov instance (inner A solve, inner SIMPLE solve, outer Schur CG).
struct CgState {
    double tol;
    int max_iter;
    int iter;
    int status;
    int first;        // 1 until the first direction update has used beta = 0
    int done;         // outer: converged / stopped; inner: unused
    int skip_next;    // outer: the S-hat solve of this iteration is skipped
    int cap;          // outer: the iteration cap was reached in this iteration
    double rho;       // r . z
    double alpha, beta;
    double zz0;       // ||z_0||^2 (inner: preconditioned residual)
    double rr0;       // outer: ||r_0||^2
    double rel;       // inner: ||z||/||z_0||; outer: ||r||/||r_0||
    double relz;      // outer: ||z||/||z_0||
    long long total;  // iterations summed over every solve of this kind in the call
};

// Defect-correction state of the mixed-precision solve.
struct Mix {
    int refine;       // refinement steps done (true residuals formed)
    int max_refine;
    int step_iter;    // FCG iterations in the current step
    int step_max;
    int stop;         // breakdown: leave every loop
    int pad;
    double rr_step0;  // ||r||^2 at the start of the step
    double factor;    // the step ends when ||r|| <= factor * ||r_step0||
    double dq;        // d.q of the last FCG direction
};

struct Ctl {
    // options (host-written before a launch)
    int precond, stop_norm, use_graph, pad0;
    double f[3];
    // loop conditions
    unsigned long long handle[kSlots];
    unsigned int cond[kSlots];
    // Krylov instances
    CgState inA, inS, out, solo, inA32, inS32, rec;
    Mix mix;
    // results
    double g_norm2, g_scale2;
    int zero_rhs, inner_status;
    double perm[3];
    double counts[5];  // unknown faces x/y/z, fluid cells, invalid mask bytes
    double n_fluid;    // fluid cells
    double big_size[kMaxBig];  // cells of each big fluid component
    long long launches;
    unsigned int ticket;
    unsigned int pad1;
    // grid barrier of the cooperative inner-solve kernels: arrivals, and a sticky flag set
    // when a wait ran past its limit
    unsigned int bar_count;
    unsigned int bar_err;
    // poll limit of one barrier wait (0: kBarrierSpins), and, for testing the bounded
    // wait, 1 + the index of a block that leaves out its barrier arrivals (0: none); both
    // are set per handle by schur_set_barrier_limit and kept across calls
    unsigned int bar_limit;
    int bar_skip;
    // per-iteration record of the outer iteration (4 doubles per iteration: alpha, beta,
    // ||r||/||r_0||, ||z||/||z_0||; NaN where a value was not formed); null: no record
    double* hist;
    int hist_cap;
    int pad2;
};

inline long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

// Slots of the per-iteration record.
enum HistSlot : int { H_ALPHA = 0, H_BETA = 1, H_REL = 2, H_RELZ = 3 };

// Record value v of outer iteration k (0-based) when it fits the record.
__device__ __forceinline__ void hist_put(Ctl* ctl, int k, int slot, double v) {
    if (ctl->hist && k >= 0 && k < ctl->hist_cap) ctl->hist[4 * (size_t)k + slot] = v;
}

// ---- device helpers ---------------------------------------------------------------

// Cell index of (x + dx, y + dy, z + dz) with periodic wrap; -1 outside a closed box.
// Offsets are at most one cell, so one wrap suffices.
__device__ __forceinline__ long long cell_at(const Dev& g, int x, int y, int z) {
    if (x < 0) { if (!g.per[0]) return -1; x += g.nx; } else if (x >= g.nx) { if (!g.per[0]) return -1; x -= g.nx; }
    if (y < 0) { if (!g.per[1]) return -1; y += g.ny; } else if (y >= g.ny) { if (!g.per[1]) return -1; y -= g.ny; }
    if (z < 0) { if (!g.per[2]) return -1; z += g.nz; } else if (z >= g.nz) { if (!g.per[2]) return -1; z -= g.nz; }
    return ((long long)z * g.ny + y) * g.nx + x;
}

__device__ __forceinline__ void axis_step(int a, int s, int& dx, int& dy, int& dz) {
    dx = (a == 0) ? s : 0;
    dy = (a == 1) ? s : 0;
    dz = (a == 2) ? s : 0;
}

__device__ __forceinline__ void count_launch(Ctl* ctl) {
    if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0 && blockIdx.x == 0 &&
        blockIdx.y == 0 && blockIdx.z == 0)
        atomicAdd((unsigned long long*)&ctl->launches, 1ull);
}

__device__ __forceinline__ void set_cond(Ctl* ctl, int slot, unsigned v) {
    ctl->cond[slot] = v;
    if (ctl->use_graph) cudaGraphSetConditional(ctl->handle[slot], v);
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    return x;
}

// Block-sum K doubles; every block writes its partial sums, and the block that finishes
// last sums all partials in a fixed order (deterministic for a fixed grid), resets the
// ticket and returns true with the totals in v[] for all its threads.  The block's
// values go through shared memory so that one warp does the additions (8 per lane, then
// a 5-step shuffle tree): on a part whose FP64 pipe retires 2 lanes per clock and SM, a
// shuffle tree in every warp would cost several times the FP64 work.  Blocks have at
// most kBlock threads, a multiple of 32.
template <int K>
__device__ __forceinline__ bool reduce_last_block(double (&v)[K], double* partials,
                                                  unsigned int* ticket) {
    __shared__ double sm[K][kBlock];
    __shared__ unsigned int s_last;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    const int lane = tid & 31, warp = tid >> 5;
    const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
    const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
#pragma unroll
    for (int k = 0; k < K; ++k) sm[k][tid] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double x = 0.0;
            for (int j = lane; j < nthr; j += 32) x += sm[k][j];
            x = warp_sum(x);
            if (lane == 0) partials[(size_t)bid * K + k] = x;
        }
        if (lane == 0) {
            __threadfence();
            unsigned prev = atomicAdd(ticket, 1u);
            s_last = (prev == nblk - 1) ? 1u : 0u;
        }
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    for (unsigned i = tid; i < nblk; i += nthr) {
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] += __ldcg(&partials[(size_t)i * K + k]);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) sm[k][tid] = acc[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double x = 0.0;
            for (int j = lane; j < nthr; j += 32) x += sm[k][j];
            x = warp_sum(x);
            if (lane == 0) acc[k] = x;
        }
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) sm[k][0] = acc[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = sm[k][0];
    if (tid == 0) *ticket = 0u;
    return true;
}

// ---- grid barrier of a cooperative launch ------------------------------------------

// Polls of one barrier wait before it gives up: the first kBarrierBusy polls spin, the
// rest sleep >= 128 ns each (a poll takes about 0.6 us in all), so the limit is about ten
// seconds: far beyond a wait between co-resident blocks (microseconds), and long enough
// for blocks that only become resident when another stream's kernel ends.
constexpr unsigned kBarrierSpins = 1u << 24;
constexpr unsigned kBarrierBusy = 1u << 10;

// Arrival at a barrier counter: a release reduction, so that the block's writes (ordered
// before it by the preceding __syncthreads) are visible to every block whose acquire load
// reads the count it contributes to.
__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// All blocks of the grid meet here (the launch is cooperative, so they are co-resident).
// ctl->bar_count counts arrivals and is zeroed before the launch; `target` is this
// block's running count of expected arrivals.  Thread 0 arrives with a release reduction
// and waits with acquire loads; the block barriers on both sides extend that ordering to
// the block's other threads (no full fences).  A wait that exceeds kBarrierSpins polls,
// or that sees another block's failure (checked every 16th poll), sets ctl->bar_err and
// returns false, and the caller leaves its loop: the kernel then ends with an error
// status instead of hanging.
__device__ __forceinline__ bool grid_barrier(Ctl* ctl, unsigned& target) {
    __shared__ unsigned s_ok;
    __syncthreads();
    target += gridDim.x;
    if (threadIdx.x == 0) {
        const unsigned limit = ctl->bar_limit ? ctl->bar_limit : kBarrierSpins;
        if ((int)blockIdx.x + 1 != ctl->bar_skip) red_release_add_u32(&ctl->bar_count, 1u);
        unsigned ok = 1u;
        for (unsigned spin = 0;; ++spin) {
            if ((int)(ld_acquire_u32(&ctl->bar_count) - target) >= 0) break;
            if ((spin & 15u) == 15u && ld_acquire_u32(&ctl->bar_err) != 0u) { ok = 0u; break; }
            if (spin >= limit) {
                atomicExch(&ctl->bar_err, 1u);
                ok = 0u;
                break;
            }
            if (spin >= kBarrierBusy) __nanosleep(128);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0u;
}

// ---- launch recorder: direct launches on a stream, or nodes of a CUDA graph -------

template <class T> struct ident { using type = T; };

class Recorder {
  public:
    // host-driven mode: kernels launch on `stream`, loops poll ctl->cond on the host
    Recorder(cudaStream_t stream, Ctl* dctl, int* next_slot)
        : stream_(stream), graph_(nullptr), dctl_(dctl), next_slot_(next_slot) {}
    // graph mode: kernels become nodes of `graph`, loops become conditional while nodes
    Recorder(cudaGraph_t graph, Ctl* dctl, int* next_slot,
             std::vector<std::pair<int, unsigned long long>>* handles)
        : stream_(nullptr), graph_(graph), dctl_(dctl), next_slot_(next_slot),
          handles_(handles) {}

    bool ok() const { return err_ == cudaSuccess; }
    cudaError_t error() const { return err_; }
    const std::string& where() const { return where_; }

    int new_slot() {
        int s = (*next_slot_)++;
        if (s >= kSlots) fail(cudaErrorInvalidValue, "out of loop slots");
        return s < kSlots ? s : kSlots - 1;
    }

    template <typename... P>
    void launch(const char* name, void (*k)(P...), dim3 grid, dim3 block,
                typename ident<P>::type... args) {
        if (!ok()) return;
        if (!graph_) {
            k<<<grid, block, 0, stream_>>>(args...);
            check(cudaGetLastError(), name);
            return;
        }
        void* ptrs[sizeof...(P) + 1] = {(void*)&args...};
        cudaKernelNodeParams p = {};
        p.func = (void*)k;
        p.gridDim = grid;
        p.blockDim = block;
        p.sharedMemBytes = 0;
        p.kernelParams = ptrs;
        cudaGraphNode_t node;
        check(cudaGraphAddKernelNode(&node, graph_, have_last_ ? &last_ : nullptr,
                                     have_last_ ? 1 : 0, &p), name);
        last_ = node;
        have_last_ = true;
    }

    // A cooperative launch (all blocks co-resident; the kernel may use grid_barrier).
    template <typename... P>
    void launch_coop(const char* name, void (*k)(P...), dim3 grid, dim3 block,
                     typename ident<P>::type... args) {
        launch_coop_smem(name, k, grid, block, 0, args...);
    }

    // ... with `smem` bytes of dynamic shared memory per block.
    template <typename... P>
    void launch_coop_smem(const char* name, void (*k)(P...), dim3 grid, dim3 block, size_t smem,
                          typename ident<P>::type... args) {
        if (!ok()) return;
        void* ptrs[sizeof...(P) + 1] = {(void*)&args...};
        if (!graph_) {
            check(cudaLaunchCooperativeKernel((const void*)k, grid, block, ptrs, smem, stream_), name);
            return;
        }
        cudaKernelNodeParams p = {};
        p.func = (void*)k;
        p.gridDim = grid;
        p.blockDim = block;
        p.sharedMemBytes = (unsigned)smem;
        p.kernelParams = ptrs;
        cudaGraphNode_t node;
        check(cudaGraphAddKernelNode(&node, graph_, have_last_ ? &last_ : nullptr,
                                     have_last_ ? 1 : 0, &p), name);
        if (!ok()) return;
        cudaLaunchAttributeValue v = {};
        v.cooperative = 1;
        check(cudaGraphKernelNodeSetAttribute(node, cudaLaunchAttributeCooperative, &v), name);
        last_ = node;
        have_last_ = true;
    }

    // while (ctl->cond[slot]) body();  -- the kernel recorded just before the loop and
    // the last kernel of the body set the condition.
    void loop(int slot, const std::function<void(Recorder&)>& body) {
        if (!ok()) return;
        if (!graph_) {
            for (;;) {
                unsigned c = 0;
                check(cudaMemcpyAsync(&c, &dctl_->cond[slot], sizeof(c), cudaMemcpyDeviceToHost,
                                      stream_), "loop condition read");
                check(cudaStreamSynchronize(stream_), "loop condition sync");
                if (!ok() || !c) break;
                body(*this);
                if (!ok()) break;
            }
            return;
        }
        cudaGraphConditionalHandle h;
        check(cudaGraphConditionalHandleCreate(&h, graph_, 0, 0), "conditional handle");
        if (!ok()) return;
        handles_->push_back({slot, (unsigned long long)h});
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        check(cudaGraphAddNode(&node, graph_, have_last_ ? &last_ : nullptr, nullptr,
                               have_last_ ? 1 : 0, &np), "conditional node");
        if (!ok()) return;
        Recorder sub(np.conditional.phGraph_out[0], dctl_, next_slot_, handles_);
        body(sub);
        if (!sub.ok()) {
            err_ = sub.err_;
            where_ = sub.where_;
            return;
        }
        last_ = node;
        have_last_ = true;
    }

  private:
    void check(cudaError_t e, const char* what) {
        if (e != cudaSuccess && err_ == cudaSuccess) {
            err_ = e;
            where_ = what;
        }
    }
    void fail(cudaError_t e, const char* what) { check(e, what); }

    cudaStream_t stream_;
    cudaGraph_t graph_;
    Ctl* dctl_;
    int* next_slot_;
    std::vector<std::pair<int, unsigned long long>>* handles_ = nullptr;
    cudaGraphNode_t last_{};
    bool have_last_ = false;
    cudaError_t err_ = cudaSuccess;
    std::string where_;
};

}  // namespace schur
