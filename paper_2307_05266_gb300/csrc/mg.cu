// Multigrid-preconditioned inner CG: an aggregation V-cycle as the preconditioner of the
// inner solves for A and for S-hat_simple (the paper preconditions them with BoomerAMG,
// Section 3.2; this is a GPU-native replacement written for the compact layout).
//
// Hierarchy (built once per geometry on the host from the device's fine tables):
//   level l + 1 merges the entries of level l whose voxel coordinates agree after halving
//   (x / 2, y / 2, z / 2; velocity components are never merged), so a 2 x 2 x 2 block is
//   one coarse unknown per component.  P is piecewise constant and A_(l+1) = P^T A_l P,
//   which stays 7-point: each coarse entry keeps one coefficient per direction (the fine
//   couplings that leave the aggregate that way) and a diagonal (its fine diagonals plus
//   the couplings that stay inside).  Levels are added until the grid is a single cell;
//   that last matrix is diagonal and is solved exactly by its pseudo-inverse.  A diagonal
//   at most 1e-12 times the entry's diagonal mass (the sum of the fine diagonals it
//   aggregates) counts as zero: the entry is a nullspace unknown with weight 0.  The
//   coefficients are summed in FP64 on the host and stored in FP32.
// V-cycle (from x = 0, on the residual r of the CG), in FP32 for both CG precisions: the
//   preconditioner only has to approximate A^-1 (its rounding perturbs the search
//   directions by about 1e-7 relative, while the CG's iterates, residual updates, dot
//   products and stop test stay in the CG's own precision).  Per level: z = omega D^-1 b
//   (formed with b), res = b - A z (one stencil on z), b_(l+1) = P^T res (a gather over the
//   8 children), the coarse correction scaled by gamma (over-correction), and one Jacobi
//   sweep after: out = y + omega D^-1 (b - A y) with y = z + gamma P out_(l+1), which the
//   parent writes into the level's res buffer once that residual is consumed.  omega = 0.9;
//   gamma = 1.3 (A) and 1.7 (S-hat).  The cycle is symmetric positive definite; the CG stop
//   rule is ||M^-1 r_k|| / ||M^-1 r_0|| < eps as for Jacobi, and the S-hat cycle's output is
//   not projected (r stays in the range; the solution is projected afterwards).
// Launch: one persistent cooperative kernel per inner solve.  The fine level and the large
//   coarse levels run on the whole grid with a grid barrier after each phase (on a coarse
//   level: the restriction, the down stencil, and on the way up the post-smoothing with the
//   prolongation); the levels from `tail` down (at most kMgTailSlots entries together) run
//   in block 0 alone, in its shared memory (the tables are copied there once per launch),
//   with block barriers, while the other blocks wait at one grid barrier.  Every grid wait
//   is bounded (grid_barrier).
#include <algorithm>
#include <atomic>
#include <cstddef>
#include <cstring>
#include <thread>
#include <type_traits>

#include "cg_dev.cuh"

namespace schur {

constexpr double kMgOmega = 0.9;
constexpr double kMgGammaA = 1.3;
constexpr double kMgGammaS = 1.7;
constexpr double kMgZeroDiag = 1e-12;
constexpr int kMgMaxLevels = 40;
// Threads per block of the loop kernel (one block per SM) for CG vectors of type T on the
// operator A (kS false) or S-hat.  The register budget per thread is 65536 / threads; with
// 1024 threads (64 registers) the kernel spills.  Measured at 128^3 (time per iteration
// against 1024 threads): FP64 A 768 threads (80 registers) -2 %, 640 +7 %, 896 +12 %;
// FP64 S-hat 640 threads -6 %; FP32 A and S-hat 896 threads (72 registers) -7 %.
template <typename T, bool kS> struct MgBlock {
    static constexpr int v = sizeof(T) == 8 ? (kS ? 640 : 768) : 896;
};
constexpr int kMgTailSlots = 2400;         // shared-memory entries of the one-block tail
constexpr int kMgMaxTail = 16;             // levels in the tail at most

// L2 prefetch distance of the fine-level phases, in grid-stride steps: 1 for FP64 CG vectors
// (measured 6 % less time per A iteration at 128^3), none for FP32 ones (no gain).
template <typename T> struct MgPrefetch { static constexpr int v = sizeof(T) == 8 ? 1 : 0; };

// Block 0's shared-memory copy of the tail levels (levels tail .. nlev-1): slot off[l] + i
// holds entry i of tail level l, slot off[l] + n_l its zero sentinel.  nb and ch hold
// level-local indices (ch: into the level below; for the first tail level, whose children
// live on a grid level, only when that level has at most 65535 entries, MgRun::ch16).  The
// tables come from a host-built image in global memory with the same layout; b, z, res
// start at zero.
struct MgTailSm {
    float b[kMgTailSlots], z[kMgTailSlots], res[kMgTailSlots];
    float dg[kMgTailSlots], wd[kMgTailSlots];
    float w[6][kMgTailSlots];
    uint16_t nb[6][kMgTailSlots];
    uint16_t ch[8][kMgTailSlots];
};
constexpr size_t kMgTailTables = offsetof(MgTailSm, dg);   // vectors come first

// Device descriptor of one level (FP32).  Every vector has one more entry, kept at 0, that
// the sentinels of the tables point at (a missing neighbour, a missing child).  Level 0: b
// is the FP32 copy of an FP64 CG residual (the kernel reads the FP32 residual it is given),
// and the operator comes from the fine tables (nb, ch, w, dg unused).  res holds the residual after pre-smoothing on the way down and, once the
// level above has consumed it, y = z + gamma P out_(l+1) on the way up.
struct MgLev {
    uint32_t n, ld, nfine;
    const uint32_t* nb;   // [6][ld] neighbour entry per direction, n = none
    const uint32_t* ch;   // [8][ld] children at level l - 1, nfine = none
    const float* w;       // [6][ld] off-diagonal coefficients (0 at missing neighbours)
    const float* dg;      // [n] diagonal
    const float* wd;      // [n + 1] omega / diagonal (0: nullspace); last level: 1 / diagonal
    float* b;             // [n + 1] right-hand side of the level
    float* z;             // [n + 1] pre-smoothed correction wd b
    float* res;           // [n + 1] residual after pre-smoothing, then y
};

struct MgRun {
    const MgLev* lev;     // [nlev] device descriptors
    const MgTailSm* img;  // tail image (tables of the tail levels)
    int nlev, tail;
    int ch16;             // the first tail level's children are in the shared-memory ch table
    float gamma;
    int off[kMgMaxTail];  // slot offset of tail level tail + k
};

// ---- per-entry work of one phase ----------------------------------------------------------

// Fine operator of the compact layout (FP32) applied at entry i to a vector v, v_i = vi.
template <bool kS>
__device__ __forceinline__ float fine_apply(const Tabs<float>& t, const Dev& g, const Compact& C,
                                            uint32_t i, float vi, const float* __restrict__ v) {
    const int ne = 2 * g.d;
    float s = 0.0f;
    if constexpr (!kS) {
        const int gh = C.ufl[i] >> 1;
#pragma unroll
        for (int e = 0; e < 6; ++e)
            if (e < ne) s += v[__ldg(C.nbA + e * C.ldA + i)];
        return t.diag[gh] * vi - s;
    } else {
        const uint32_t code = __ldg(C.codeS + i);
#pragma unroll
        for (int e = 0; e < 6; ++e)
            if (e < ne) s += t.w[(code >> (3 * e)) & 7u] * (vi - v[__ldg(C.nbS + e * C.ldS + i)]);
        return s;
    }
}

// Coarse operator of a level (fields of its descriptor) applied at entry i to v.
__device__ __forceinline__ float coarse_apply(const uint32_t* __restrict__ nb, const float* __restrict__ w,
                                              const float* __restrict__ dg, uint32_t ld, uint32_t i,
                                              float vi, const float* __restrict__ v) {
    float s = dg[i] * vi;
#pragma unroll
    for (int e = 0; e < 6; ++e) s += w[e * ld + i] * v[__ldg(nb + e * ld + i)];
    return s;
}

// b at entry i of a level: the sum of its children's residuals.
__device__ __forceinline__ float restrict_at(const uint32_t* __restrict__ ch, uint32_t ld,
                                             const float* __restrict__ resf, uint32_t i) {
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += resf[__ldg(ch + c * ld + i)];
    return s;
}

// Prolongation of the correction `out` of entry i of level L to its children: y = z + gamma
// out on the level below F (written into F's res buffer, whose residual is consumed).
__device__ __forceinline__ void prolong_entry(const MgLev* __restrict__ L, const MgLev* __restrict__ F,
                                              float gamma, float out, uint32_t i) {
    const uint32_t* __restrict__ ch = L->ch;
    const uint32_t ld = L->ld, nf = L->nfine;
    const float* __restrict__ zf = F->z;
    float* __restrict__ yf = F->res;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const uint32_t k = __ldg(ch + c * ld + i);
        if (k < nf) yf[k] = zf[k] + gamma * out;
    }
}

// Fine-level stencil phase over the whole grid, U entries per thread and step with all of
// their loads issued before the arithmetic (the gathers are latency-bound).  Down:
// res0 = b0 - Op z0.  Up: the cycle's output y + wd0 (b0 - Op y), y = res0, handed to
// emit(i, value).
template <bool kS, bool kUp, int U, int PF, class Emit>
__device__ __forceinline__ void fine_phase(const Tabs<float>& t, const Dev& g, const Compact& C,
                                           const MgLev* __restrict__ L, const float* __restrict__ b,
                                           uint32_t n, Emit emit) {
    const float* __restrict__ v = kUp ? L->res : L->z;
    float* __restrict__ res = L->res;
    const float* __restrict__ wd = L->wd;
    const int ne = 2 * g.d;
    const uint32_t* __restrict__ nbt = kS ? C.nbS : C.nbA;
    const long long ldt = kS ? C.ldS : C.ldA;
    WARP_STREAM_BEGIN_U(n, U)
        if constexpr (PF > 0) {   // the streamed operands of a later step, into L2
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const uint32_t k = idx[j] + PF * step_;
                if (k < n) {
#pragma unroll
                    for (int e = 0; e < 6; ++e)
                        if (e < ne) prefetch_l2(nbt + e * ldt + k);
                    if constexpr (kS) prefetch_l2(C.codeS + k);
                    else prefetch_l2(C.ufl + k);
                    prefetch_l2(v + k);
                    prefetch_l2(b + k);
                    if constexpr (kUp) prefetch_l2(wd + k);
                }
            }
        }
        uint32_t nb[U][6], key[U];
        float vc[U], bc[U], wc[U];
#pragma unroll
        for (int j = 0; j < U; ++j)
            if (idx[j] < n) {
#pragma unroll
                for (int e = 0; e < 6; ++e) nb[j][e] = e < ne ? __ldg(nbt + e * ldt + idx[j]) : n;
                if constexpr (kS) key[j] = __ldg(C.codeS + idx[j]);
                else key[j] = C.ufl[idx[j]];
                vc[j] = v[idx[j]];
                bc[j] = b[idx[j]];
                if constexpr (kUp) wc[j] = wd[idx[j]];
            }
#pragma unroll
        for (int j = 0; j < U; ++j)
            if (idx[j] < n) {
                float sv[6];
#pragma unroll
                for (int e = 0; e < 6; ++e) sv[e] = v[nb[j][e]];
                float a;
                if constexpr (!kS) {
                    a = t.diag[key[j] >> 1] * vc[j] - (((sv[0] + sv[1]) + (sv[2] + sv[3])) + (sv[4] + sv[5]));
                } else {
                    a = 0.0f;
#pragma unroll
                    for (int e = 0; e < 6; ++e) a += t.w[(key[j] >> (3 * e)) & 7u] * (vc[j] - sv[e]);
                }
                if constexpr (kUp) emit(idx[j], vc[j] + wc[j] * (bc[j] - a));
                else res[idx[j]] = bc[j] - a;
            }
    WARP_STREAM_END
}

// Coarse level, restriction alone over a loop: b = P^T res_(l-1), z = wd b.
#define MG_RESTRICT(LOOP, Lp, Fp)                                                           \
    {                                                                                       \
        const uint32_t* __restrict__ ch_ = (Lp)->ch;                                        \
        const uint32_t ld_ = (Lp)->ld, n_ = (Lp)->n;                                        \
        const float* __restrict__ resf_ = (Fp)->res;                                        \
        const float* __restrict__ wd_ = (Lp)->wd;                                           \
        float* __restrict__ b_ = (Lp)->b;                                                   \
        float* __restrict__ z_ = (Lp)->z;                                                   \
        LOOP(i, n_) {                                                                       \
            const float bi = restrict_at(ch_, ld_, resf_, i);                               \
            b_[i] = bi;                                                                     \
            z_[i] = wd_[i] * bi;                                                            \
        }                                                                                   \
    }

// Coarse level, down stencil alone: res = b - A z.
#define MG_DOWN(LOOP, Lp)                                                                   \
    {                                                                                       \
        const uint32_t* __restrict__ nb_ = (Lp)->nb;                                        \
        const float* __restrict__ w_ = (Lp)->w;                                             \
        const float* __restrict__ dg_ = (Lp)->dg;                                           \
        const uint32_t ld_ = (Lp)->ld, n_ = (Lp)->n;                                        \
        const float* __restrict__ z_ = (Lp)->z;                                             \
        const float* __restrict__ b_ = (Lp)->b;                                             \
        float* __restrict__ res_ = (Lp)->res;                                               \
        LOOP(i, n_) res_[i] = b_[i] - coarse_apply(nb_, w_, dg_, ld_, i, z_[i], z_);        \
    }

// Coarse level, up: out = y + wd (b - A y), prolonged to the level below.
#define MG_UP(LOOP, Lp, Fp, gamma)                                                          \
    {                                                                                       \
        const uint32_t* __restrict__ nb_ = (Lp)->nb;                                        \
        const float* __restrict__ w_ = (Lp)->w;                                             \
        const float* __restrict__ dg_ = (Lp)->dg;                                           \
        const float* __restrict__ wd_ = (Lp)->wd;                                           \
        const uint32_t ld_ = (Lp)->ld, n_ = (Lp)->n;                                        \
        const float* __restrict__ y_ = (Lp)->res;                                           \
        const float* __restrict__ b_ = (Lp)->b;                                             \
        LOOP(i, n_) {                                                                       \
            const float yi = y_[i];                                                         \
            const float out = yi + wd_[i] * (b_[i] - coarse_apply(nb_, w_, dg_, ld_, i, yi, y_)); \
            prolong_entry((Lp), (Fp), (gamma), out, i);                                     \
        }                                                                                   \
    }

// ---- loops over a level: the whole grid (grid-stride) or block 0 alone -----------------

#define MG_GRID_LOOP(i, n)                                                                  \
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += gridDim.x * blockDim.x)
#define MG_BLOCK_LOOP(i, n) for (uint32_t i = threadIdx.x; i < (n); i += blockDim.x)

// ---- the tail: levels tail .. nlev-1 in block 0's shared memory -----------------------

// Copies the tail tables into shared memory and zeroes its vectors (block 0, once per launch).
__device__ __forceinline__ void tail_load(MgTailSm& T, const MgTailSm* __restrict__ img) {
    const uint32_t* src = (const uint32_t*)((const char*)img + kMgTailTables);
    uint32_t* dst = (uint32_t*)((char*)&T + kMgTailTables);
    const int nw = (int)((sizeof(MgTailSm) - kMgTailTables) / 4);
    for (int k = threadIdx.x; k < nw; k += blockDim.x) dst[k] = __ldg(src + k);
    float* v = (float*)&T;
    for (int k = threadIdx.x; k < 3 * kMgTailSlots; k += blockDim.x) v[k] = 0.0f;
    __syncthreads();
}

// One pass of the tail levels: restriction from the grid level tail - 1, down to the exact
// solve of the last level, and back up to the prolongation into level tail - 1.
__device__ __forceinline__ void tail_cycle(MgTailSm& T, const MgRun& M, const MgLev* lev) {
    const int t = M.tail, nlev = M.nlev;
    const float gamma = M.gamma;
    for (int l = t; l < nlev; ++l) {
        const MgLev* __restrict__ L = lev + l;
        const uint32_t n = L->n;
        const int o = M.off[l - t];
        if (l == t && M.ch16) {   // restriction from the grid level below (global memory)
            // two entries per thread and step, so that both sets of gathers are in flight
            // together; an entry past the end reads the sentinel slot (children = the zero
            // entry of the level below) and is not stored
            const float* __restrict__ resf = lev[l - 1].res;
            for (uint32_t i = threadIdx.x; i < n; i += 2 * blockDim.x) {
                const uint32_t i2 = i + blockDim.x;
                const int k1 = o + (int)i, k2 = o + (int)(i2 < n ? i2 : n);
                float b1 = 0.0f, b2 = 0.0f;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    b1 += resf[T.ch[c][k1]];
                    b2 += resf[T.ch[c][k2]];
                }
                T.b[k1] = b1;
                T.z[k1] = T.wd[k1] * b1;
                if (i2 < n) {
                    T.b[k2] = b2;
                    T.z[k2] = T.wd[k2] * b2;
                }
            }
        } else if (l == t) {
            const float* __restrict__ resf = lev[l - 1].res;
            MG_BLOCK_LOOP(i, n) {
                const float b = restrict_at(L->ch, L->ld, resf, i);
                T.b[o + i] = b;
                T.z[o + i] = T.wd[o + i] * b;
            }
        } else {
            const int of = M.off[l - 1 - t];
            MG_BLOCK_LOOP(i, n) {
                float b = 0.0f;
#pragma unroll
                for (int c = 0; c < 8; ++c) b += T.res[of + T.ch[c][o + i]];
                T.b[o + i] = b;
                T.z[o + i] = T.wd[o + i] * b;
            }
        }
        __syncthreads();
        if (l == nlev - 1) break;   // z of the last level is its exact solve
        MG_BLOCK_LOOP(i, n) {
            const int k = o + i;
            float s = T.dg[k] * T.z[k];
#pragma unroll
            for (int e = 0; e < 6; ++e) s += T.w[e][k] * T.z[o + T.nb[e][k]];
            T.res[k] = T.b[k] - s;
        }
        __syncthreads();
    }
    // up: the correction of level l (its exact solve on the last level, else the post-
    // smoothed y) prolonged into the level below
    for (int l = nlev - 1; l >= t; --l) {
        const MgLev* __restrict__ L = lev + l;
        const uint32_t n = L->n;
        const int o = M.off[l - t];
        MG_BLOCK_LOOP(i, n) {
            const int k = o + i;
            float out;
            if (l == nlev - 1) {
                out = T.z[k];
            } else {
                const float y = T.res[k];
                float s = T.dg[k] * y;
#pragma unroll
                for (int e = 0; e < 6; ++e) s += T.w[e][k] * T.res[o + T.nb[e][k]];
                out = y + T.wd[k] * (T.b[k] - s);
            }
            if (l > t) {
                const int of = M.off[l - 1 - t];
                const uint32_t nf = L->nfine;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const uint32_t kk = T.ch[c][k];
                    if (kk < nf) T.res[of + kk] = T.z[of + kk] + gamma * out;
                }
            } else if (M.ch16) {
                const MgLev* __restrict__ F = lev + (l - 1);
                const uint32_t nf = L->nfine;
                const float* __restrict__ zf = F->z;
                float* __restrict__ yf = F->res;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const uint32_t kk = T.ch[c][k];
                    if (kk < nf) yf[kk] = zf[kk] + gamma * out;
                }
            } else {
                prolong_entry(L, lev + (l - 1), gamma, out, i);
            }
        }
        __syncthreads();
    }
}

// The multigrid-preconditioned CG loop of one inner solve in precision T, after its init
// kernel (x = 0, r = b, status NOTCONV when b != 0).  r32: the FP32 copy of r that the cycle
// reads (r itself when T is float).  dS: the diagonal of S-hat (FP64 S stencil).  Same
// contract as the Jacobi loop kernels: all blocks hold bitwise-equal scalars (block-
// identical grid sums), `gate` skips the solve, block 0 writes the final state, a failed
// barrier leaves ST_BARRIER.
template <typename T, bool kS>
__device__ __forceinline__ void mg_loop(const Dev& g, const Compact& C, const MgRun& M,
                                        const T* __restrict__ dS, T* __restrict__ xv,
                                        T* __restrict__ rv, T* __restrict__ pv, T* __restrict__ qv,
                                        float* __restrict__ r32, Ctl* ctl, CgState* st,
                                        double* partials, const int* gate) {
    constexpr bool kSame = std::is_same<T, float>::value;
    constexpr int PF = MgPrefetch<T>::v;
    constexpr int NT = MgBlock<T, kS>::v;
    // FP64 CG vectors: the cycle's output z stays FP32 (exact in T) in the level-0 z buffer,
    // half the bytes of q; FP32 ones: z in q.
    constexpr bool kZ32 = !kSame;
    __shared__ CgState s;
    __shared__ unsigned s_cont;
    __shared__ Tabs<T> t;
    __shared__ Tabs<float> tf;
    // the level descriptors, copied once per launch: every phase starts from its level's
    // fields, and a global load there would put one dependent round trip before each phase
    __shared__ MgLev lev[kMgMaxLevels];
    extern __shared__ __align__(16) unsigned char mg_dyn[];
    MgTailSm& tsm = *reinterpret_cast<MgTailSm*>(mg_dyn);
    if (gate && *gate) return;
    {
        static_assert(sizeof(MgLev) % 4 == 0, "descriptor copy by 32-bit words");
        const uint32_t* src = reinterpret_cast<const uint32_t*>(M.lev);
        uint32_t* dst = reinterpret_cast<uint32_t*>(lev);
        const int nw = M.nlev * (int)(sizeof(MgLev) / 4);
        for (int k = threadIdx.x; k < nw; k += blockDim.x) dst[k] = __ldg(src + k);
    }
    load_tabs<T>(g, t);
    load_tabs<float>(g, tf);
    if (blockIdx.x == 0) tail_load(tsm, M.img);
    if (threadIdx.x == 0) s = *st;
    __syncthreads();
    if (s.status != ST_NOTCONV || ld_acquire_u32(&ctl->bar_err) != 0u) return;
    const uint32_t n = (uint32_t)(kS ? C.n_p : C.n_u);
    double* P1 = partials;               // [grid] p.q
    double* P2 = partials + kMaxBlocks;  // [grid][2] r.z, z.z
    const int tail = M.tail;
    const float gamma = M.gamma;
    unsigned target = 0;
    bool ok = true;
    bool started = false;
    // The step x += alpha p of an iteration is taken in the next cycle, by the blocks that
    // wait at the grid barrier while block 0 runs the tail levels: nothing in the cycle
    // reads x, and p keeps its value until the direction phase after the cycle.
    T alpha_prev = (T)0;   // the step x += alpha_prev p not yet taken
    {   // the FP32 residual and z0 = wd0 r for the first cycle (later: with the r update)
        const float* __restrict__ wd0 = lev[0].wd;
        float* __restrict__ z0 = lev[0].z;
        MG_GRID_LOOP(i, n) {
            const float ri = (float)rv[i];
            if constexpr (!kSame) r32[i] = ri;
            z0[i] = wd0[i] * ri;
        }
    }
    for (;;) {
        // ---- V-cycle on r (r32 and z0 complete after this barrier)
        if (!(ok = grid_barrier(ctl, target))) break;
        fine_phase<kS, false, 1, PF>(tf, g, C, lev, r32, n, [](uint32_t, float) {});
        if (!(ok = grid_barrier(ctl, target))) break;
        for (int l = 1; l < tail; ++l) {
            const MgLev* __restrict__ L = lev + l;
            const MgLev* __restrict__ F = lev + (l - 1);
            MG_RESTRICT(MG_GRID_LOOP, L, F);
            if (!(ok = grid_barrier(ctl, target))) break;
            MG_DOWN(MG_GRID_LOOP, L);
            if (!(ok = grid_barrier(ctl, target))) break;
        }
        if (!ok) break;
        if (blockIdx.x == 0) tail_cycle(tsm, M, lev);
        if (alpha_prev != (T)0 && (blockIdx.x > 0 || gridDim.x == 1)) {
            // x += alpha_prev p: blocks 1 .. grid - 1 (block 0 alone on a one-block grid)
            const T ap = alpha_prev;
            T* __restrict__ x = opaque(xv);
            const T* __restrict__ p = opaque(pv);
            const uint32_t nb = gridDim.x > 1 ? gridDim.x - 1 : 1u;
            const uint32_t b = gridDim.x > 1 ? blockIdx.x - 1 : 0u;
            const uint32_t stride = nb * blockDim.x;
            const uint32_t ahead = PF * stride;
            for (uint32_t i = b * blockDim.x + threadIdx.x; i < n; i += stride) {
                if (PF > 0 && i + ahead < n) {
                    prefetch_l2(x + i + ahead);
                    prefetch_l2(p + i + ahead);
                }
                x[i] += ap * p[i];
            }
        }
        alpha_prev = (T)0;
        if (!(ok = grid_barrier(ctl, target))) break;
        for (int l = tail - 1; l >= 1; --l) {
            const MgLev* __restrict__ L = lev + l;
            const MgLev* __restrict__ F = lev + (l - 1);
            MG_UP(MG_GRID_LOOP, L, F, gamma);
            if (!(ok = grid_barrier(ctl, target))) break;
        }
        if (!ok) break;
        // ---- z = the cycle's output, r.z and z.z.  kZ32: z is an FP32 value (exact in T),
        // kept in the level-0 z buffer (z0 was consumed by the prolongation into level 0
        // above and is formed again by the update below); else in q
        double v2[2];
        {
            T a0 = (T)0, a1 = (T)0;
            float* __restrict__ zout = lev[0].z;
            T* __restrict__ q = qv;
            const T* __restrict__ r = rv;
            fine_phase<kS, true, 1, PF>(tf, g, C, lev, r32, n, [&](uint32_t i, float zf32) {
                const T zf = (T)zf32;
                if constexpr (kZ32) zout[i] = zf32;
                else q[i] = zf;
                a0 += r[i] * zf;
                a1 += zf * zf;
            });
            v2[0] = (double)a0;
            v2[1] = (double)a1;
        }
        if (!(ok = grid_sum<2, NT>(v2, P2, ctl, target))) break;
        // the first cycle of the kernel starts the iteration (rho, ||z_0||); every later one
        // ends an iteration (count, stop test, beta)
        if (threadIdx.x == 0) {
            s_cont = started ? finish_inner(nullptr, &s, v2[0], v2[1])
                             : start_inner(nullptr, &s, v2[0], v2[1]);
        }
        __syncthreads();
        started = true;
        if (!s_cont) break;
        // ---- p = z + beta p
        if constexpr (kZ32) {
            const T beta = (T)(s.first ? 0.0 : s.beta);
            T* __restrict__ p = opaque(pv);
            const float* __restrict__ z = opaque(lev[0].z);
            const uint32_t ahead = PF * gridDim.x * blockDim.x;
            MG_GRID_LOOP(i, n) {
                if (PF > 0 && i + ahead < n) {
                    prefetch_l2(z + i + ahead);
                    prefetch_l2(p + i + ahead);
                }
                p[i] = (T)z[i] + beta * p[i];
            }
        } else {
            const T beta = (T)(s.first ? 0.0 : s.beta);
            T* __restrict__ p = opaque(pv);
            const T* __restrict__ z = opaque(qv);
            MG_GRID_LOOP(i, n) p[i] = z[i] + beta * p[i];
        }
        if (!(ok = grid_barrier(ctl, target))) break;
        // ---- q = Op p, p.q
        double v1[1];
        {
            Compact Cl = C;
            Cl.nbA = opaque(C.nbA);
            Cl.nbS = opaque(C.nbS);
            Cl.codeS = opaque(C.codeS);
            Cl.ufl = opaque(C.ufl);
            // one entry per thread and step: in this 64-register kernel the two-entry form of
            // the Jacobi loops spills (measured 7 % more time per FP64 A iteration at 128^3)
            constexpr int U = 1;
            if constexpr (kS)
                v1[0] = (double)phaseS_matvec<T, U>(t, g, Cl, opaque(dS), opaque(pv), opaque(qv));
            else
                v1[0] = (double)phaseA_matvec<T, U>(t, g, Cl, opaque(pv), opaque(qv));
        }
        if (!(ok = grid_sum<1, NT>(v1, P1, ctl, target))) break;
        if (threadIdx.x == 0) {
            s_cont = matvec_alpha(&s, v1[0]) ? 1u : 0u;
            if (!s_cont) finish_inner(nullptr, &s, 0.0, 0.0);  // counts the iteration
        }
        __syncthreads();
        if (!s_cont) break;
        // ---- r -= alpha q, the FP32 residual and z0 = wd0 r (x += alpha p: next cycle)
        {
            const T alpha = (T)s.alpha;
            T* __restrict__ r = opaque(rv);
            const T* __restrict__ q = opaque(qv);
            const float* __restrict__ w0 = opaque(lev[0].wd);
            float* __restrict__ z0 = opaque(lev[0].z);
            float* __restrict__ rf = opaque(r32);
            const uint32_t ahead = PF * gridDim.x * blockDim.x;
            MG_GRID_LOOP(i, n) {
                if (PF > 0 && i + ahead < n) {
                    const uint32_t k = i + ahead;
                    prefetch_l2(r + k);
                    prefetch_l2(q + k);
                    prefetch_l2(w0 + k);
                }
                const T ri = r[i] - alpha * q[i];
                r[i] = ri;
                const float r32i = (float)ri;
                if constexpr (!kSame) rf[i] = r32i;
                z0[i] = w0[i] * r32i;
            }
            alpha_prev = alpha;
        }
    }
    // a step x += alpha p still due (the loop ends after a cycle, which has taken it, so this
    // is a safeguard; p is unchanged since its update phase, and the kernel ends here)
    if (ok && alpha_prev != (T)0) {
        const T ap = alpha_prev;
        T* __restrict__ x = opaque(xv);
        const T* __restrict__ p = opaque(pv);
        MG_GRID_LOOP(i, n) x[i] += ap * p[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (!ok) s.status = ST_BARRIER;
        *st = s;
        note_inner_status(ctl, s.status);
    }
}

template <typename T, bool kS>
__global__ void __launch_bounds__(MgBlock<T, kS>::v, 1) k_mg_loop(Dev g, Compact C, MgRun M,
                                                       const T* __restrict__ dS, T* __restrict__ xv,
                                                       T* __restrict__ rv, T* __restrict__ pv,
                                                       T* __restrict__ qv, float* __restrict__ r32,
                                                       Ctl* ctl, CgState* st, double* partials,
                                                       const int* gate) {
    count_launch(ctl);
    mg_loop<T, kS>(g, C, M, dS, xv, rv, pv, qv, r32, ctl, st, partials, gate);
}

// ---- hierarchy build (host) ---------------------------------------------------------------

namespace {

// Host threads of the hierarchy build.  Every parallel step writes disjoint entries, and each
// coarse sum keeps the serial order of its terms, so the hierarchy does not depend on the
// thread count.
int host_threads() {
    const unsigned hw = std::thread::hardware_concurrency();
    return (int)std::max(1u, std::min(hw ? hw : 1u, 16u));
}

// fn(t, begin, end) for the ranges [cut[t], cut[t + 1]), one thread each (the last on the
// calling thread).  When a thread cannot be had, the ranges left run on the calling thread:
// no exception leaves the library.  fn itself allocates nothing.
template <class Fn>
void run_ranges(const std::vector<long long>& cut, Fn fn) {
    const int nt = (int)cut.size() - 1;
    std::vector<std::thread> th;
    int t = 0;
    try {
        th.reserve((size_t)std::max(nt - 1, 0));
        for (; t + 1 < nt; ++t) th.emplace_back(fn, t, cut[t], cut[t + 1]);
    } catch (...) {
    }
    for (; t < nt; ++t) fn(t, cut[t], cut[t + 1]);
    for (auto& x : th) x.join();
}

// nt equal ranges of [0, n).
std::vector<long long> cuts(long long n, int nt) {
    nt = (int)std::max(1ll, std::min<long long>(nt, n));
    std::vector<long long> cut((size_t)nt + 1);
    for (int t = 0; t <= nt; ++t) cut[t] = n * t / nt;
    return cut;
}

// Equal ranges of [0, n) for the host threads (a single range below 2^16 entries).
std::vector<long long> even_cuts(long long n) { return cuts(n, n < (1 << 16) ? 1 : host_threads()); }

// One level on the host: coordinates (component a, voxel x, y, z of the level's grid), the
// 7-point couplings and the diagonal with its mass.  The fine level keeps the device's own
// neighbour table (row stride ld, sentinel n) and derives its coefficients: -1 per unknown
// neighbour for A' (wmode UNIT), -1 / (2d + g) per open face for S-hat (wmode CODE, from
// the 3-bit face codes); coarse levels store theirs (wmode TABLE).
struct HostLevel {
    enum { TABLE, UNIT, CODE } wmode = TABLE;
    long long n = 0, ld = 0;
    int dims[3] = {1, 1, 1};
    std::vector<int8_t> a;
    std::vector<int16_t> x, y, z;
    std::vector<uint32_t> nb;     // [6][ld], n = none
    std::vector<double> w;        // [6][ld] (TABLE)
    std::vector<uint32_t> code;   // [n] (CODE)
    double wcode[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    std::vector<double> dg, mass;

    double coef(int e, long long i) const {
        if (wmode == TABLE) return w[e * ld + i];
        if (wmode == UNIT) return -1.0;
        return -wcode[(code[i] >> (3 * e)) & 7u];
    }
};

template <typename T>
cudaError_t mg_alloc(MgOp& M, cudaStream_t s, T** p, size_t n) {
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return e;
    }
    M.bufs.push_back((void*)*p);
    M.bytes += (long long)(n * sizeof(T));
    return cudaMemsetAsync(*p, 0, n * sizeof(T), s);
}

// Copy a host vector to a new device buffer on stream s (waits: the vector is temporary).
template <typename T>
cudaError_t upload(MgOp& M, cudaStream_t s, T** dst, const std::vector<T>& src) {
    cudaError_t e = mg_alloc(M, s, dst, src.size());
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
}

template <typename T>
cudaError_t download(cudaStream_t s, const T* src, size_t n, std::vector<T>& out) {
    out.resize(n);
    if (!n) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(out.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
}

// Fine level of A' = h^2 A or of S-hat from the device tables of the compact layout.
cudaError_t fine_level(const Handle& H, bool simple, HostLevel& L) {
    const Dev& g = H.g;
    const long long n = simple ? H.n_p : H.n_u;
    L.n = n;
    L.ld = simple ? H.ldS : H.ldA;
    L.dims[0] = g.nx;
    L.dims[1] = g.ny;
    L.dims[2] = g.nz;
    std::vector<uint32_t> idx;
    cudaError_t e = download(H.stream, simple ? H.flist : H.ulist, (size_t)n, idx);
    if (e == cudaSuccess)
        e = download(H.stream, simple ? H.nbS : H.nbA, (size_t)(2 * g.d * L.ld), L.nb);
    if (e != cudaSuccess) return e;
    L.nb.resize((size_t)(6 * L.ld), (uint32_t)n);   // 2D: the z rows are empty
    L.a.resize(n);
    L.x.resize(n);
    L.y.resize(n);
    L.z.resize(n);
    const long long plane = (long long)g.nx * g.ny;
    run_ranges(even_cuts(n), [&](int, long long k0, long long k1) {
        for (long long k = k0; k < k1; ++k) {
            long long i = idx[k];
            int a = 0;
            if (!simple) {
                a = (int)(i / g.stride);
                i -= (long long)a * g.stride;
            }
            const long long zz = i / plane, rem = i - zz * plane;
            L.a[k] = (int8_t)a;
            L.z[k] = (int16_t)zz;
            L.y[k] = (int16_t)(rem / g.nx);
            L.x[k] = (int16_t)(rem - (rem / g.nx) * g.nx);
        }
    });
    if (!simple) {
        std::vector<uint8_t> ufl;
        if ((e = download(H.stream, H.ufl, (size_t)n, ufl)) != cudaSuccess) return e;
        L.wmode = HostLevel::UNIT;
        L.dg.resize(n);
        for (long long k = 0; k < n; ++k) L.dg[k] = g.diag[ufl[k] >> 1];
    } else {
        if ((e = download(H.stream, H.codeS, (size_t)n, L.code)) != cudaSuccess) return e;
        if ((e = download(H.stream, H.dSc, (size_t)n, L.dg)) != cudaSuccess) return e;
        L.wmode = HostLevel::CODE;
        for (int c = 1; c < 6; ++c) L.wcode[c] = g.wdiag[c - 1];
    }
    L.mass = L.dg;
    return cudaSuccess;
}

// The next level of F: parent of every entry of F, the coarse coordinates, children,
// neighbour table and Galerkin coefficients.  Returns false when a fine coupling leaves its
// aggregate towards an aggregate that is not the coarse neighbour in that direction.
bool coarsen(const HostLevel& F, const int per[3], int ncomp, HostLevel& C,
             std::vector<uint32_t>& agg, std::vector<uint32_t>& ch) {
    const int cx = (F.dims[0] + 1) / 2, cy = (F.dims[1] + 1) / 2, cz = (F.dims[2] + 1) / 2;
    const long long cells = (long long)cx * cy * cz;
    std::vector<int32_t> idx((size_t)(ncomp * cells), -1);
    auto key = [&](int a, int X, int Y, int Z) {
        return ((long long)a * cz + Z) * cy * cx + (long long)Y * cx + X;
    };
    // F is ordered by (a, z, y, x), so the entries of one coarse slab (a, z / 2) are
    // contiguous: ranges cut at slab boundaries own disjoint sets of aggregates
    std::vector<long long> cut = even_cuts(F.n);
    for (size_t t = 1; t + 1 < cut.size(); ++t) {
        long long i = std::max(cut[t], cut[t - 1]);
        while (i > 0 && i < F.n && F.a[i] == F.a[i - 1] && (F.z[i] >> 1) == (F.z[i - 1] >> 1)) ++i;
        cut[t] = i;
    }
    run_ranges(cut, [&](int, long long i0, long long i1) {
        for (long long i = i0; i < i1; ++i) idx[key(F.a[i], F.x[i] >> 1, F.y[i] >> 1, F.z[i] >> 1)] = 0;
    });
    // coarse entries in (a, Z, Y, X) order: counts per slab, their prefix sums, numbering
    const long long nslab = (long long)ncomp * cz, slab = (long long)cx * cy;
    std::vector<long long> cnt((size_t)nslab + 1, 0);
    const std::vector<long long> scut = cuts(nslab, nslab * slab < (1 << 16) ? 1 : host_threads());
    run_ranges(scut, [&](int, long long s0, long long s1) {
        for (long long sl = s0; sl < s1; ++sl) {
            long long c = 0;
            for (long long k = sl * slab; k < (sl + 1) * slab; ++k) c += idx[k] >= 0;
            cnt[sl + 1] = c;
        }
    });
    for (long long sl = 0; sl < nslab; ++sl) cnt[sl + 1] += cnt[sl];
    const long long nc = cnt[nslab];
    C = HostLevel();
    C.dims[0] = cx;
    C.dims[1] = cy;
    C.dims[2] = cz;
    C.n = nc;
    C.a.resize(nc);
    C.x.resize(nc);
    C.y.resize(nc);
    C.z.resize(nc);
    run_ranges(scut, [&](int, long long s0, long long s1) {
        for (long long sl = s0; sl < s1; ++sl) {
            long long v = cnt[sl];
            const int a = (int)(sl / cz), Z = (int)(sl % cz);
            for (int Y = 0; Y < cy; ++Y)
                for (int X = 0; X < cx; ++X) {
                    int32_t& e = idx[key(a, X, Y, Z)];
                    if (e < 0) continue;
                    e = (int32_t)v;
                    C.a[v] = (int8_t)a;
                    C.x[v] = (int16_t)X;
                    C.y[v] = (int16_t)Y;
                    C.z[v] = (int16_t)Z;
                    ++v;
                }
        }
    });
    C.ld = round_up(nc + 1, 32);
    agg.assign((size_t)F.n + 1, (uint32_t)nc);
    ch.assign((size_t)(8 * C.ld), (uint32_t)F.n);
    run_ranges(cut, [&](int, long long i0, long long i1) {
        for (long long i = i0; i < i1; ++i) {
            const uint32_t I = (uint32_t)idx[key(F.a[i], F.x[i] >> 1, F.y[i] >> 1, F.z[i] >> 1)];
            agg[i] = I;
            const int slot = (F.x[i] & 1) | ((F.y[i] & 1) << 1) | ((F.z[i] & 1) << 2);
            ch[slot * C.ld + I] = (uint32_t)i;
        }
    });
    // coarse neighbours: the aggregate one step away along each direction (wrapped on a
    // periodic axis); a step that wraps onto the aggregate itself is a diagonal coupling
    const int cd[3] = {cx, cy, cz};
    C.nb.assign((size_t)(6 * C.ld), (uint32_t)nc);
    run_ranges(even_cuts(nc), [&](int, long long I0, long long I1) {
        for (long long I = I0; I < I1; ++I)
            for (int e = 0; e < 6; ++e) {
                const int b = e >> 1, sgn = (e & 1) ? 1 : -1;
                int c3[3] = {C.x[I], C.y[I], C.z[I]};
                c3[b] += sgn;
                if (c3[b] < 0 || c3[b] >= cd[b]) {
                    if (!per[b]) continue;
                    c3[b] = (c3[b] + cd[b]) % cd[b];
                }
                const int32_t J = idx[key(C.a[I], c3[0], c3[1], c3[2])];
                if (J >= 0 && J != I) C.nb[e * C.ld + I] = (uint32_t)J;
            }
    });
    // Galerkin coefficients, each summed over its fine entries in their order (the slab
    // ranges own their aggregates)
    C.w.assign((size_t)(6 * C.ld), 0.0);
    C.dg.assign((size_t)nc, 0.0);
    C.mass.assign((size_t)nc, 0.0);
    std::atomic<bool> consistent(true);
    run_ranges(cut, [&](int, long long i0, long long i1) {
        for (long long i = i0; i < i1; ++i) {
            const uint32_t I = agg[i];
            C.dg[I] += F.dg[i];
            C.mass[I] += F.mass[i];
            for (int e = 0; e < 6; ++e) {
                const uint32_t j = F.nb[e * F.ld + i];
                if (j >= (uint32_t)F.n) continue;
                const double c = F.coef(e, i);
                const uint32_t J = agg[j];
                if (J == I) {
                    C.dg[I] += c;
                } else {
                    if (C.nb[e * C.ld + I] != J) {
                        consistent = false;
                        return;
                    }
                    C.w[e * C.ld + I] += c;
                }
            }
        }
    });
    return consistent;
}

bool single_cell(const HostLevel& L) {
    for (long long i = 0; i < L.n; ++i)
        if (L.x[i] || L.y[i] || L.z[i]) return false;
    return true;
}

// Weights of the smoother (omega / diagonal) or, on the last level, of the exact solve
// (1 / diagonal); 0 for a diagonal that counts as zero; one more entry (0) for the sentinel.
std::vector<float> weights(const HostLevel& L, double scale) {
    std::vector<float> wd((size_t)L.n + 1, 0.0f);
    for (long long i = 0; i < L.n; ++i)
        if (L.dg[i] > kMgZeroDiag * L.mass[i]) wd[i] = (float)(scale / L.dg[i]);
    return wd;
}

std::vector<float> to_float(const std::vector<double>& v) {
    return std::vector<float>(v.begin(), v.end());
}

int build_hierarchy(Handle& H, MgOp& M, bool simple) {
    const Dev& g = H.g;
    const cudaStream_t s = H.stream;
    cudaError_t e = cudaStreamSynchronize(s);   // the fine tables are complete
    const int ncomp = simple ? 1 : g.d;
    std::vector<HostLevel> lv(1);
    if (e == cudaSuccess) e = fine_level(H, simple, lv[0]);
    if (e != cudaSuccess) return schur_set_error_internal(SCHUR_ECUDA, cudaGetErrorString(e));
    std::vector<std::vector<uint32_t>> chs(1);
    do {   // at least one coarse level, until the grid is a single cell
        HostLevel c;
        std::vector<uint32_t> agg, ch;
        if (!coarsen(lv.back(), g.per, ncomp, c, agg, ch))
            return schur_set_error_internal(SCHUR_ECUDA, "multigrid: inconsistent coarse coupling");
        chs.push_back(std::move(ch));
        lv.push_back(std::move(c));
    } while (!single_cell(lv.back()) && (int)lv.size() < kMgMaxLevels);
    if (!single_cell(lv.back()))
        return schur_set_error_internal(SCHUR_EINVAL, "multigrid: too many levels");
    for (double v : lv.back().w)
        if (v != 0.0) return schur_set_error_internal(SCHUR_ECUDA, "multigrid: last level not diagonal");
    const int L = (int)lv.size();
    M.nlev = L;
    M.n.assign(L, 0);
    // tail: the largest set of last levels whose entries (and one sentinel each) fit the
    // shared-memory slots, with 16-bit level-local indices (level 0 stays on the grid)
    M.tail = L;
    {
        long long slots = 0;
        for (int l = L - 1; l >= 1 && L - l <= kMgMaxTail; --l) {
            slots += lv[l].n + 1;
            if (slots > kMgTailSlots || lv[l].n >= 65535) break;
            M.tail = l;
        }
    }
    if (M.tail >= L)
        return schur_set_error_internal(SCHUR_EINVAL, "multigrid: last level too large");
    // the first tail level's children as 16-bit indices when the grid level below has at
    // most 65535 entries (its sentinel index included)
    M.ch16 = lv[M.tail - 1].n <= 65535 ? 1 : 0;
    {   // the tail image: tables of the tail levels in their shared-memory layout
        std::vector<MgTailSm> img(1);
        std::memset(img.data(), 0, sizeof(MgTailSm));
        MgTailSm& T = img[0];
        int o = 0;
        M.off.clear();
        for (int l = M.tail; l < L; ++l) {
            const HostLevel& v = lv[l];
            M.off.push_back(o);
            const bool last = (l == L - 1);
            const std::vector<float> wd = weights(v, last ? 1.0 : kMgOmega);
            for (long long i = 0; i <= v.n; ++i) {
                const int k = o + (int)i;
                for (int e = 0; e < 6; ++e) T.nb[e][k] = (uint16_t)v.n;
                const bool has_ch = l > M.tail || M.ch16;
                for (int c = 0; c < 8; ++c) T.ch[c][k] = (uint16_t)(has_ch ? lv[l - 1].n : 0);
                if (i == v.n) continue;
                T.dg[k] = (float)v.dg[i];
                T.wd[k] = wd[i];
                for (int e = 0; e < 6; ++e) {
                    T.nb[e][k] = (uint16_t)v.nb[e * v.ld + i];
                    T.w[e][k] = (float)v.w[e * v.ld + i];
                }
                if (has_ch)
                    for (int c = 0; c < 8; ++c) T.ch[c][k] = (uint16_t)chs[l][c * v.ld + i];
            }
            o += (int)v.n + 1;
        }
        MgTailSm* dimg = nullptr;
        e = upload(M, s, &dimg, img);
        M.img = dimg;
    }
    std::vector<MgLev> d((size_t)L);
    for (int l = 0; l < L && e == cudaSuccess; ++l) {
        const HostLevel& v = lv[l];
        M.n[l] = v.n;
        MgLev& dl = d[l];
        std::memset(&dl, 0, sizeof(dl));
        dl.n = (uint32_t)v.n;
        dl.ld = (uint32_t)v.ld;
        dl.nfine = l > 0 ? (uint32_t)lv[l - 1].n : 0u;
        const bool last = (l == L - 1);
        float *wd = nullptr, *w = nullptr, *dg = nullptr;
        uint32_t *nb = nullptr, *ch = nullptr;
        e = upload(M, s, &wd, weights(v, last ? 1.0 : kMgOmega));
        if (e == cudaSuccess && l == 0) e = mg_alloc(M, s, &dl.b, (size_t)v.n + 1);  // FP64 CG: r32
        if (e == cudaSuccess && l > 0) e = upload(M, s, &nb, v.nb);
        if (e == cudaSuccess && l > 0) e = upload(M, s, &ch, chs[l]);
        if (e == cudaSuccess && l > 0) e = upload(M, s, &w, to_float(v.w));
        if (e == cudaSuccess && l > 0) e = upload(M, s, &dg, to_float(v.dg));
        if (e == cudaSuccess && l > 0) e = mg_alloc(M, s, &dl.b, (size_t)v.n + 1);
        if (e == cudaSuccess) e = mg_alloc(M, s, &dl.z, (size_t)v.n + 1);
        if (e == cudaSuccess) e = mg_alloc(M, s, &dl.res, (size_t)v.n + 1);
        dl.wd = wd;
        dl.w = w;
        dl.dg = dg;
        dl.nb = nb;
        dl.ch = ch;
    }
    if (e == cudaSuccess) {
        M.r32 = d[0].b;
        MgLev* dev = nullptr;
        e = mg_alloc(M, s, &dev, (size_t)L);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dev, d.data(), (size_t)L * sizeof(MgLev), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        M.lev = dev;
    }
    if (e == cudaErrorMemoryAllocation)
        return schur_set_error_internal(SCHUR_ENOMEM, "device allocation failed");
    if (e != cudaSuccess) return schur_set_error_internal(SCHUR_ECUDA, cudaGetErrorString(e));
    return SCHUR_OK;
}

}  // namespace

void mg_free(MgOp& M) {
    for (void* p : M.bufs) cudaFree(p);
    M = MgOp();
}

int mg_prepare(Handle& H, bool simple) {
    MgOp& M = simple ? H.mgS : H.mgA;
    if ((simple ? H.n_p : H.n_u) == 0 || M.nlev) return SCHUR_OK;
    const int rc = build_hierarchy(H, M, simple);
    if (rc) {
        mg_free(M);
        return rc;
    }
    H.bytes += M.bytes;
    return SCHUR_OK;
}

// Grid of a multigrid loop kernel of `nt` threads per block: one block per SM at most (the
// kernel's resident blocks with its shared memory, and the launch shape's cap), at least
// one block per nt x 4 entries; allows the kernel's dynamic shared memory first.
template <class K>
static dim3 mg_grid(const Handle& H, long long n, K k, size_t smem, int nt) {
    static std::mutex mu;
    {
        std::lock_guard<std::mutex> lock(mu);
        cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    const long long res = (long long)H.nsm * resident_blocks((const void*)k, smem, nt);
    const long long shape = std::max<long long>(1, H.target_blocks / 8);   // blocks_per_sm x nsm / 8
    const long long want = std::max<long long>(std::min<long long>(H.nsm, (n + nt - 1) / nt),
                                               (n + 4LL * nt - 1) / (4LL * nt));
    return dim3((unsigned)std::max<long long>(1, std::min(std::min(res, shape), want)));
}

void record_mg_loop(Handle& H, Recorder& R, bool simple, bool fp32, void* x, void* r, void* p,
                    void* q, CgState* st, const int* gate) {
    const MgOp& M = simple ? H.mgS : H.mgA;
    const Compact C = compact_of(H);
    const long long n = simple ? H.n_p : H.n_u;
    if (!M.nlev) return;   // no entries: the init kernel already finished the solve
    MgRun run;
    std::memset(&run, 0, sizeof(run));
    run.lev = (const MgLev*)M.lev;
    run.img = (const MgTailSm*)M.img;
    run.nlev = M.nlev;
    run.tail = M.tail;
    run.ch16 = M.ch16;
    run.gamma = (float)(simple ? kMgGammaS : kMgGammaA);
    for (size_t k = 0; k < M.off.size() && k < (size_t)kMgMaxTail; ++k) run.off[k] = M.off[k];
    const size_t sm = sizeof(MgTailSm);
    constexpr int ntAd = MgBlock<double, false>::v, ntSd = MgBlock<double, true>::v;
    constexpr int ntAf = MgBlock<float, false>::v, ntSf = MgBlock<float, true>::v;
    if (!fp32) {
        // the cycle reads an FP32 copy of the FP64 residual
        if (simple)
            R.launch_coop_smem("mgS_loop", k_mg_loop<double, true>, mg_grid(H, n, k_mg_loop<double, true>, sm, ntSd),
                               dim3(ntSd), sm, H.g, C, run, (const double*)H.dSc, (double*)x, (double*)r,
                               (double*)p, (double*)q, M.r32, H.dctl, st, H.partials, gate);
        else
            R.launch_coop_smem("mgA_loop", k_mg_loop<double, false>, mg_grid(H, n, k_mg_loop<double, false>, sm, ntAd),
                               dim3(ntAd), sm, H.g, C, run, (const double*)nullptr, (double*)x, (double*)r,
                               (double*)p, (double*)q, M.r32, H.dctl, st, H.partials, gate);
    } else {
        // FP32 CG: the cycle reads the residual itself (its level-0 descriptor points at r32,
        // which the kernel does not touch)
        if (simple)
            R.launch_coop_smem("mgS_loop_f32", k_mg_loop<float, true>, mg_grid(H, n, k_mg_loop<float, true>, sm, ntSf),
                               dim3(ntSf), sm, H.g, C, run, (const float*)nullptr, (float*)x, (float*)r,
                               (float*)p, (float*)q, (float*)r, H.dctl, st, H.partials, gate);
        else
            R.launch_coop_smem("mgA_loop_f32", k_mg_loop<float, false>, mg_grid(H, n, k_mg_loop<float, false>, sm, ntAf),
                               dim3(ntAf), sm, H.g, C, run, (const float*)nullptr, (float*)x, (float*)r,
                               (float*)p, (float*)q, (float*)r, H.dctl, st, H.partials, gate);
    }
}

}  // namespace schur
