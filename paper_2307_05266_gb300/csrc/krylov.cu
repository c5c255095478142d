// Krylov kernels and the recorded control flow of a solve.
//
// Inner solves: Jacobi-preconditioned CG from x_0 = 0 with the stopping rule of
// Section 3.2, ||M^-1 r_k|| / ||M^-1 r_0|| < eps, for A (face space, M = diag(A)) and
// for S-hat_simple (cell space, M = diag(S-hat)).  One CG iteration is three kernels:
//   dir:    p = z + beta p  (z = M^-1 r formed on the fly; beta = 0 on the first pass)
//   matvec: q = Op p and the partial sums of p.q; the last block forms alpha = rho/p.q
//   update: x += alpha p, r -= alpha q, partial sums of r.z and z.z; the last block
//           forms beta, tests convergence and sets the loop condition.
// The inner kernels are templates on the storage/arithmetic type T: FP64 for the plain
// path, FP32 for the mixed-precision path (GB300 runs FP32 at 64x its FP64 rate).  Dot
// products are summed per thread in T and across threads and blocks in FP64.
// Outer solve, FP64: Algorithm 1 with r = g - S p (the printed sign of r^0 and of the r
// update is inconsistent; standard PCG of Saad Alg. 9.1 is used), p_0 = 0, and either
// the unpreconditioned ||r_k||/||r_0|| or the preconditioned ||z_k||/||z_0|| stop.
// Mixed precision: FP64 flexible CG (Notay's FCG(1): beta = -z.q_prev / d.q_prev,
// alpha = d.r / d.q) over FP32 inner solves, inside FP64 defect correction: each
// refinement step runs FCG on S delta = r until ||r|| drops by a fixed factor, then
// recomputes the true residual r = g - S p with FP64 inner solves.
// All scalars live in the device control block; every loop is a conditional while node
// of one CUDA graph (or a host loop in debugging mode).  Every loop terminates: each
// condition update either continues below its iteration cap or stops.
#include <cmath>

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

template <typename T>
__device__ __forceinline__ double face_val(const Dev& g, const uint8_t* __restrict__ flags,
                                           const T* __restrict__ u, int a, int x, int y, int z) {
    long long c = cell_at(g, x, y, z);
    if (c < 0) return 0.0;
    const long long i = (long long)a * g.stride + c;
    return (flags[i] & 1) ? (double)u[i] : 0.0;
}

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
    if (st > ctl->inner_status) ctl->inner_status = st;
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

__device__ __forceinline__ void finish_matvec(Ctl* ctl, CgState* st, double dq, int slot) {
    if (!(dq > 0.0) || isinf(dq)) {
        st->status = ST_BREAKDOWN;
        st->alpha = 0.0;
        set_cond(ctl, slot, 0u);
    } else {
        st->alpha = st->rho / dq;
    }
}

// ------------------------------------------------------------------------------------
// access patterns
// ------------------------------------------------------------------------------------
// Streaming kernels walk compact work lists (unknown faces, fluid cells): a warp owns
// kU chunks of 32 list entries per step (lane l takes entry base + l + 32 j), so each
// thread has kU independent gathers in flight and every lane does useful work.  Faces
// that are not unknowns and solid cells hold 0 in every solver vector from allocation
// on and are never read or written.
constexpr int kU = 4;

#define WARP_STREAM_BEGIN(n)                                                              \
    {                                                                                     \
        const long long lane_ = threadIdx.x & 31;                                         \
        const long long nw_ = ((long long)gridDim.x * blockDim.x) >> 5;                   \
        for (long long base_ = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5)  \
                               * (32 * kU);                                               \
             base_ < (n); base_ += nw_ * (32 * kU)) {                                     \
            long long idx[kU];                                                            \
            _Pragma("unroll") for (int j = 0; j < kU; ++j) idx[j] = base_ + lane_ + 32 * j;
#define WARP_STREAM_END \
        }               \
    }

// Column tiles (used once per inner solve): x-y tiles strided over blockIdx.x,
// gridDim.y = z chunks, blockIdx.z = component.
#define COLUMN_TILES_BEGIN(g)                                                         \
    const int gx_ = ((g).nx + kTileX - 1) / kTileX;                                   \
    const int gy_ = ((g).ny + kTileY - 1) / kTileY;                                   \
    const int zc_ = ((g).nz + gridDim.y - 1) / gridDim.y;                             \
    const int z0_ = blockIdx.y * zc_;                                                 \
    const int z1_ = min((g).nz, z0_ + zc_);                                           \
    const long long plane = (long long)(g).nx * (g).ny;                               \
    for (int t_ = blockIdx.x; t_ < gx_ * gy_; t_ += gridDim.x) {                      \
        const int x = (t_ % gx_) * kTileX + (int)threadIdx.x;                         \
        const int y = (t_ / gx_) * kTileY + (int)threadIdx.y;                         \
        if (x < (g).nx && y < (g).ny) {                                               \
            const long long cxy = (long long)y * (g).nx + x;                          \
            for (int z = z0_; z < z1_; ++z) {                                         \
                const long long c = z * plane + cxy;
#define COLUMN_TILES_END \
            }            \
        }                \
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

// ------------------------------------------------------------------------------------
// inner CG on A (face space)
// ------------------------------------------------------------------------------------
// The inner A solve works with the dimensionless operator A' = h^2 A (diagonal 2d + g,
// off-diagonal -1) and M' = diag(A'), right-hand side h^2 b: alpha, beta and every
// iterate x are those of CG on A x = b with Jacobi M = diag(A), without h^-2 factors.

// b = cf f_a + cp h^-1 (P_c - P_(c-e_a)) (+ bvec) on unknown faces (formed in FP64);
// x = 0, r = h^2 b.
template <typename T>
__global__ void k_cgA_init(Dev g, const uint8_t* __restrict__ flags, T* __restrict__ xv,
                           T* __restrict__ rv, const double* __restrict__ P, double cp,
                           double cf, const double* __restrict__ bvec, Ctl* ctl, CgState* st,
                           double* partials, int slot) {
    count_launch(ctl);
    double v[2] = {0.0, 0.0};
    const int a = blockIdx.z;
    const uint8_t* F = flags + (long long)a * g.stride;
    const long long lower = a == 0 ? 1 : (a == 1 ? g.nx : (long long)g.nx * g.ny);
    const double fa = cf * ctl->f[a];
    COLUMN_TILES_BEGIN(g)
        const uint8_t f = F[c];
        if (f & 1) {
            // an unknown face has a fluid lower cell inside the box (wrap when periodic)
            long long cl = c - lower;
            if ((a == 0 && x == 0) || (a == 1 && y == 0) || (a == 2 && z == 0))
                cl += (a == 0 ? g.nx : (a == 1 ? (long long)g.ny * g.nx : (long long)g.nz * plane));
            double b = fa;
            if (P) b += cp * (g.hinv * (P[c] - P[cl]));
            const long long i = (long long)a * g.stride + c;
            if (bvec) b += bvec[i];
            const T bt = (T)(b * g.h2);  // right-hand side of h^2 A x = h^2 b
            const double bd = (double)bt;
            const double zz = bd * tab5(g.wdiag, f >> 1);
            v[0] += bd * zz;
            v[1] += zz * zz;
            xv[i] = (T)0;
            rv[i] = bt;
        }
    COLUMN_TILES_END
    if (reduce_last_block<2>(v, partials, &ctl->ticket) && is_thread0())
        set_cond(ctl, slot, start_inner(ctl, st, v[0], v[1]));
}

// p = M'^-1 r + beta p over the unknown-face list.
template <typename T>
__global__ void k_cgA_dir(Dev g, const uint32_t* __restrict__ list, long long n,
                          const uint8_t* __restrict__ flags, const T* __restrict__ rv,
                          T* __restrict__ pv, Ctl* ctl, const CgState* st) {
    count_launch(ctl);
    const T beta = (T)(st->first ? 0.0 : st->beta);
    WARP_STREAM_BEGIN(n)
        uint32_t i[kU];
        int gh[kU];
        T r[kU], p[kU];
#pragma unroll
        for (int j = 0; j < kU; ++j) i[j] = idx[j] < n ? list[idx[j]] : 0u;
#pragma unroll
        for (int j = 0; j < kU; ++j)
            if (idx[j] < n) { gh[j] = flags[i[j]] >> 1; r[j] = rv[i[j]]; p[j] = pv[i[j]]; }
#pragma unroll
        for (int j = 0; j < kU; ++j)
            if (idx[j] < n) pv[i[j]] = r[j] * Tab<T>::w(g, gh[j]) + beta * p[j];
    WARP_STREAM_END
}

// q = A' p and p.q over the unknown-face list; neighbours that are not unknowns hold 0.
template <typename T>
__global__ void k_cgA_matvec(Dev g, const uint32_t* __restrict__ list, long long n,
                             const uint8_t* __restrict__ flags, const T* __restrict__ pv,
                             T* __restrict__ qv, Ctl* ctl, CgState* st, double* partials,
                             int slot) {
    count_launch(ctl);
    T acc = (T)0;
    const long long plane = (long long)g.nx * g.ny;
    STREAM_LOOP(k, n) {
        const uint32_t i = list[k];
        const FaceAt f = decode_face(g, i);
        const int gh = flags[i] >> 1;
        const T* P = pv + (long long)f.a * g.stride;
        const long long c = f.c;
        const T pc = P[c];
        const long long xm = f.x > 0 ? c - 1 : (g.per[0] ? c + g.nx - 1 : -1);
        const long long xp = f.x < g.nx - 1 ? c + 1 : (g.per[0] ? c - (g.nx - 1) : -1);
        const long long ym = f.y > 0 ? c - g.nx : (g.per[1] ? c + (long long)(g.ny - 1) * g.nx : -1);
        const long long yp = f.y < g.ny - 1 ? c + g.nx : (g.per[1] ? c - (long long)(g.ny - 1) * g.nx : -1);
        T s = (xm >= 0 ? P[xm] : (T)0) + (xp >= 0 ? P[xp] : (T)0);
        s += (ym >= 0 ? P[ym] : (T)0) + (yp >= 0 ? P[yp] : (T)0);
        if (g.d == 3) {
            const long long zm = f.z > 0 ? c - plane : (g.per[2] ? c + (long long)(g.nz - 1) * plane : -1);
            const long long zp = f.z < g.nz - 1 ? c + plane : (g.per[2] ? c - (long long)(g.nz - 1) * plane : -1);
            s += (zm >= 0 ? P[zm] : (T)0) + (zp >= 0 ? P[zp] : (T)0);
        }
        const T out = Tab<T>::diag(g, gh) * pc - s;
        qv[i] = out;
        acc += pc * out;
    }
    double v[1] = {(double)acc};
    if (reduce_last_block<1>(v, partials, &ctl->ticket) && is_thread0())
        finish_matvec(ctl, st, v[0], slot);
}

// x += alpha p, r -= alpha q; r.z and z.z (z = M'^-1 r) over the unknown-face list.
template <typename T>
__global__ void k_cgA_update(Dev g, const uint32_t* __restrict__ list, long long n,
                             const uint8_t* __restrict__ flags, T* __restrict__ xv,
                             T* __restrict__ rv, const T* __restrict__ pv,
                             const T* __restrict__ qv, Ctl* ctl, CgState* st,
                             double* partials, int slot) {
    count_launch(ctl);
    const T alpha = (T)st->alpha;
    T a0 = (T)0, a1 = (T)0;
    WARP_STREAM_BEGIN(n)
        uint32_t i[kU];
        int gh[kU];
        T xx[kU], p[kU], r[kU], q[kU];
#pragma unroll
        for (int j = 0; j < kU; ++j) i[j] = idx[j] < n ? list[idx[j]] : 0u;
#pragma unroll
        for (int j = 0; j < kU; ++j)
            if (idx[j] < n) {
                gh[j] = flags[i[j]] >> 1;
                xx[j] = xv[i[j]];
                p[j] = pv[i[j]];
                r[j] = rv[i[j]];
                q[j] = qv[i[j]];
            }
#pragma unroll
        for (int j = 0; j < kU; ++j)
            if (idx[j] < n) {
                xv[i[j]] = xx[j] + alpha * p[j];
                const T rn = r[j] - alpha * q[j];
                rv[i[j]] = rn;
                const T zz = rn * Tab<T>::w(g, gh[j]);
                a0 += rn * zz;
                a1 += zz * zz;
            }
    WARP_STREAM_END
    double v[2] = {(double)a0, (double)a1};
    if (reduce_last_block<2>(v, partials, &ctl->ticket) && is_thread0())
        set_cond(ctl, slot, finish_inner(ctl, st, v[0], v[1]));
}

// ------------------------------------------------------------------------------------
// inner CG on S-hat_simple (cell space); M^-1 = invd (0 on solid and isolated cells)
// ------------------------------------------------------------------------------------

// b = r - (its mean on r's fluid component): the FP64 outer residual r is projected onto
// the range of S-hat in place, then x = 0 and the CG residual starts at b.
template <typename T>
__global__ void k_cgS_init(Dev g, const T* __restrict__ invd, const int* __restrict__ cmp,
                           const double* __restrict__ cmean, double* __restrict__ b,
                           T* __restrict__ xv, T* __restrict__ rv, Ctl* ctl, CgState* st,
                           const CgState* outer, double* partials, int slot) {
    count_launch(ctl);
    if (outer->skip_next) {
        if (blockIdx.x == 0 && is_thread0()) set_cond(ctl, slot, 0u);
        return;
    }
    double v[2] = {0.0, 0.0};
    STREAM_LOOP(c, g.ncell) {
        const int k = cmp[c];
        if (k >= 0) {
            const double bc = b[c] - cmean[k];
            b[c] = bc;
            const T bt = (T)bc;
            const double zz = (double)bt * (double)invd[c];
            v[0] += (double)bt * zz;
            v[1] += zz * zz;
            xv[c] = (T)0;
            rv[c] = bt;
        }
    }
    if (reduce_last_block<2>(v, partials, &ctl->ticket) && is_thread0())
        set_cond(ctl, slot, start_inner(ctl, st, v[0], v[1]));
}

template <typename T>
__global__ void k_cgS_dir(Dev g, const uint32_t* __restrict__ list, long long n,
                          const T* __restrict__ invd, const T* __restrict__ rv,
                          T* __restrict__ pv, Ctl* ctl, const CgState* st) {
    count_launch(ctl);
    const T beta = (T)(st->first ? 0.0 : st->beta);
    WARP_STREAM_BEGIN(n)
        uint32_t i[kU];
        T r[kU], w[kU], p[kU];
#pragma unroll
        for (int j = 0; j < kU; ++j) i[j] = idx[j] < n ? list[idx[j]] : 0u;
#pragma unroll
        for (int j = 0; j < kU; ++j)
            if (idx[j] < n) { r[j] = rv[i[j]]; w[j] = invd[i[j]]; p[j] = pv[i[j]]; }
#pragma unroll
        for (int j = 0; j < kU; ++j)
            if (idx[j] < n) pv[i[j]] = r[j] * w[j] + beta * p[j];
    WARP_STREAM_END
}

// q = S-hat p and p.q over the fluid-cell list: the sum over the open faces of
// (p_c - p_nb) / (2d + g_f).
template <typename T>
__global__ void k_cgS_matvec(Dev g, const uint32_t* __restrict__ list, long long n,
                             const uint8_t* __restrict__ flags, const T* __restrict__ pv,
                             T* __restrict__ qv, Ctl* ctl, CgState* st, double* partials,
                             int slot) {
    count_launch(ctl);
    T acc = (T)0;
    const long long plane = (long long)g.nx * g.ny;
    const uint8_t* F0 = flags;
    const uint8_t* F1 = flags + g.stride;
    const uint8_t* F2 = flags + 2 * g.stride;
    STREAM_LOOP(k, n) {
        const uint32_t ci = list[k];
        const FaceAt f = decode_face(g, ci);
        const long long c = f.c;
        const T pc = pv[c];
        T out = (T)0;
        // lower faces: an unknown lower face has its lower cell inside the box
        uint8_t fl = F0[c];
        if (fl & 1) out += (pc - pv[f.x > 0 ? c - 1 : c + g.nx - 1]) * Tab<T>::w(g, fl >> 1);
        fl = F1[c];
        if (fl & 1) out += (pc - pv[f.y > 0 ? c - g.nx : c + (long long)(g.ny - 1) * g.nx]) * Tab<T>::w(g, fl >> 1);
        // upper faces
        const long long xp = f.x < g.nx - 1 ? c + 1 : (g.per[0] ? c - (g.nx - 1) : -1);
        if (xp >= 0) { fl = F0[xp]; if (fl & 1) out += (pc - pv[xp]) * Tab<T>::w(g, fl >> 1); }
        const long long yp = f.y < g.ny - 1 ? c + g.nx : (g.per[1] ? c - (long long)(g.ny - 1) * g.nx : -1);
        if (yp >= 0) { fl = F1[yp]; if (fl & 1) out += (pc - pv[yp]) * Tab<T>::w(g, fl >> 1); }
        if (g.d == 3) {
            fl = F2[c];
            if (fl & 1) out += (pc - pv[f.z > 0 ? c - plane : c + (long long)(g.nz - 1) * plane]) * Tab<T>::w(g, fl >> 1);
            const long long zp = f.z < g.nz - 1 ? c + plane : (g.per[2] ? c - (long long)(g.nz - 1) * plane : -1);
            if (zp >= 0) { fl = F2[zp]; if (fl & 1) out += (pc - pv[zp]) * Tab<T>::w(g, fl >> 1); }
        }
        qv[c] = out;
        acc += pc * out;
    }
    double v[1] = {(double)acc};
    if (reduce_last_block<1>(v, partials, &ctl->ticket) && is_thread0())
        finish_matvec(ctl, st, v[0], slot);
}

template <typename T>
__global__ void k_cgS_update(Dev g, const uint32_t* __restrict__ list, long long n,
                             const T* __restrict__ invd, T* __restrict__ xv,
                             T* __restrict__ rv, const T* __restrict__ pv,
                             const T* __restrict__ qv, Ctl* ctl, CgState* st,
                             double* partials, int slot) {
    count_launch(ctl);
    const T alpha = (T)st->alpha;
    T a0 = (T)0, a1 = (T)0;
    WARP_STREAM_BEGIN(n)
        uint32_t i[kU];
        T xx[kU], p[kU], r[kU], q[kU], w[kU];
#pragma unroll
        for (int j = 0; j < kU; ++j) i[j] = idx[j] < n ? list[idx[j]] : 0u;
#pragma unroll
        for (int j = 0; j < kU; ++j)
            if (idx[j] < n) {
                xx[j] = xv[i[j]];
                p[j] = pv[i[j]];
                r[j] = rv[i[j]];
                q[j] = qv[i[j]];
                w[j] = invd[i[j]];
            }
#pragma unroll
        for (int j = 0; j < kU; ++j)
            if (idx[j] < n) {
                xv[i[j]] = xx[j] + alpha * p[j];
                const T rn = r[j] - alpha * q[j];
                rv[i[j]] = rn;
                const T zz = rn * w[j];
                a0 += rn * zz;
                a1 += zz * zz;
            }
    WARP_STREAM_END
    double v[2] = {(double)a0, (double)a1};
    if (reduce_last_block<2>(v, partials, &ctl->ticket) && is_thread0())
        set_cond(ctl, slot, finish_inner(ctl, st, v[0], v[1]));
}

// ------------------------------------------------------------------------------------
// per-component means (nullspace of S-hat_simple and S: constants per fluid component)
// ------------------------------------------------------------------------------------

// Means of v over the (at most kMaxBig) big components, summed by the whole grid.
template <typename T>
__global__ void k_comp_big(Dev g, const int* __restrict__ cmp, const T* __restrict__ v,
                           double* __restrict__ cmean, int nbig, Ctl* ctl,
                           const CgState* outer, double* partials) {
    count_launch(ctl);
    if (outer->skip_next) return;
    double s[kMaxBig];
#pragma unroll
    for (int b = 0; b < kMaxBig; ++b) s[b] = 0.0;
    STREAM_LOOP(c, g.ncell) {
        const int k = cmp[c];
        if (k >= 0 && k < nbig) {
            const double vc = (double)v[c];
#pragma unroll
            for (int b = 0; b < kMaxBig; ++b) s[b] += (k == b) ? vc : 0.0;
        }
    }
    if (reduce_last_block<kMaxBig>(s, partials, &ctl->ticket) && is_thread0()) {
        for (int b = 0; b < nbig; ++b) cmean[b] = s[b] / ctl->big_size[b];
    }
}

// Means of v over the small components, one warp per component (cells in fixed order).
template <typename T>
__global__ void k_comp_small(const int* __restrict__ start, const int* __restrict__ cells,
                             const T* __restrict__ v, double* __restrict__ cmean, int nbig,
                             int nsmall, Ctl* ctl, const CgState* outer) {
    count_launch(ctl);
    if (outer->skip_next) return;
    const int lane = threadIdx.x & 31;
    const int warps = blockDim.x >> 5;
    for (long long j = (long long)blockIdx.x * warps + (threadIdx.x >> 5); j < nsmall;
         j += (long long)gridDim.x * warps) {
        const int b0 = start[j], b1 = start[j + 1];
        double s = 0.0;
        for (int i = b0 + lane; i < b1; i += 32) s += (double)v[cells[i]];
        s = warp_sum(s);
        if (lane == 0) cmean[nbig + j] = s / (double)(b1 - b0);
    }
}

// ------------------------------------------------------------------------------------
// outer Schur CG (Algorithm 1), cell space, FP64
// ------------------------------------------------------------------------------------

// g = B u (u = A^-1 f); r = g, p = 0, d = g; zero-RHS test.
template <typename TX>
__global__ void k_outer_init(Dev g, const uint8_t* __restrict__ mask, const uint8_t* __restrict__ flags,
                             const TX* __restrict__ u, double* __restrict__ gv,
                             double* __restrict__ rv, double* __restrict__ pv,
                             double* __restrict__ dv, Ctl* ctl, double* partials, int slot) {
    count_launch(ctl);
    double v[2] = {0.0, 0.0};
    TILE_LOOP_BEGIN(g)
        double gc = 0.0;
        if (mask[c] == 1) {
            double s = 0.0, sa = 0.0;
            for (int a = 0; a < g.d; ++a) {
                int ex, ey, ez;
                axis_step(a, 1, ex, ey, ez);
                const double up = face_val(g, flags, u, a, x + ex, y + ey, z + ez);
                const double lo = face_val(g, flags, u, a, x, y, z);
                s += up - lo;
                sa += fabs(up) + fabs(lo);
            }
            gc = -g.hinv * s;
            v[0] += gc * gc;
            v[1] += (g.hinv * sa) * (g.hinv * sa);
        }
        gv[c] = gc;
        rv[c] = gc;
        pv[c] = 0.0;
        dv[c] = gc;
    TILE_LOOP_END
    if (reduce_last_block<2>(v, partials, &ctl->ticket) && is_thread0()) {
        ctl->g_norm2 = v[0];
        ctl->g_scale2 = v[1];
        const int zero = (v[0] == 0.0) || (sqrt(v[0]) <= kZeroRhsRtol * sqrt(v[1]));
        ctl->zero_rhs = zero;
        CgState* o = &ctl->out;
        o->iter = 0;
        o->status = ST_OK;
        o->rr0 = v[0];
        o->rho = v[0];
        o->zz0 = v[0];
        o->alpha = o->beta = 0.0;
        o->done = zero;
        o->skip_next = zero;
        o->cap = 0;
        o->rel = zero ? 0.0 : 1.0;
        o->relz = zero ? 0.0 : 1.0;
        ctl->mix.refine = 0;
        ctl->mix.stop = 0;
        set_cond(ctl, slot, zero ? 0u : 1u);
    }
}

// SIMPLE: z_0 = S-hat^-1 r_0 minus its component means; d = z_0, rho = r.z, ||z_0||^2.
template <typename TX>
__global__ void k_outer_start(Dev g, const int* __restrict__ cmp, const double* __restrict__ cmean,
                              const TX* __restrict__ sx, const double* __restrict__ rv,
                              double* __restrict__ dv, Ctl* ctl, double* partials, int slot) {
    count_launch(ctl);
    if (ctl->out.done) return;
    double v[2] = {0.0, 0.0};
    STREAM_LOOP(c, g.ncell) {
        const int k = cmp[c];
        const double zc = (k >= 0) ? (double)sx[c] - cmean[k] : 0.0;
        dv[c] = zc;
        v[0] += rv[c] * zc;
        v[1] += zc * zc;
    }
    if (reduce_last_block<2>(v, partials, &ctl->ticket) && is_thread0()) {
        CgState* o = &ctl->out;
        o->rho = v[0];
        o->zz0 = v[1];
        if (v[1] == 0.0) {
            o->done = 1;
            o->skip_next = 1;
            o->relz = 0.0;
            set_cond(ctl, slot, 0u);
        }
    }
}

// q = B u with u = A^-1 B^T d; alpha = rho / d.q.
template <typename TX>
__global__ void k_outer_div(Dev g, const uint8_t* __restrict__ mask, const uint8_t* __restrict__ flags,
                            const TX* __restrict__ u, const double* __restrict__ dv,
                            double* __restrict__ qv, Ctl* ctl, double* partials, int slot) {
    count_launch(ctl);
    double v[1] = {0.0};
    TILE_LOOP_BEGIN(g)
        double qc = 0.0;
        if (mask[c] == 1) {
            double s = 0.0;
            for (int a = 0; a < g.d; ++a) {
                int ex, ey, ez;
                axis_step(a, 1, ex, ey, ez);
                s += face_val(g, flags, u, a, x + ex, y + ey, z + ez) - face_val(g, flags, u, a, x, y, z);
            }
            qc = -g.hinv * s;
            v[0] += dv[c] * qc;
        }
        qv[c] = qc;
    TILE_LOOP_END
    if (reduce_last_block<1>(v, partials, &ctl->ticket) && is_thread0()) {
        CgState* o = &ctl->out;
        const double dq = v[0];
        if (!(dq > 0.0) || isinf(dq)) {
            o->status = ST_BREAKDOWN;
            o->alpha = 0.0;
            o->done = 1;
            o->skip_next = 1;
            o->iter += 1;
            set_cond(ctl, slot, 0u);
        } else {
            o->alpha = o->rho / dq;
        }
    }
}

// p += alpha d, r -= alpha q, ||r||; unpreconditioned test; Uzawa: beta.
__global__ void k_outer_update(Dev g, double* __restrict__ pv, double* __restrict__ rv,
                               const double* __restrict__ dv, const double* __restrict__ qv,
                               Ctl* ctl, double* partials, int slot) {
    count_launch(ctl);
    CgState* o = &ctl->out;
    if (o->done) return;
    const double alpha = o->alpha;
    double v[1] = {0.0};
    STREAM_LOOP(c, g.ncell) {
        pv[c] += alpha * dv[c];
        const double r = rv[c] - alpha * qv[c];
        rv[c] = r;
        v[0] += r * r;
    }
    if (reduce_last_block<1>(v, partials, &ctl->ticket) && is_thread0()) {
        o->iter += 1;
        o->total += 1;
        const double rel = sqrt(v[0] / o->rr0);
        o->rel = rel;
        unsigned cont = 1u;
        if (ctl->stop_norm == 0 && rel < o->tol) {
            o->status = ST_OK;
            o->relz = nan("");
            cont = 0u;
        } else if (ctl->precond == 0) {
            // Uzawa: z = r
            o->relz = sqrt(v[0] / o->zz0);
            if (ctl->stop_norm == 1 && o->relz < o->tol) {
                o->status = ST_OK;
                cont = 0u;
            } else if (!(rel == rel)) {
                o->status = ST_BREAKDOWN;
                cont = 0u;
            } else if (o->iter >= o->max_iter) {
                o->status = ST_NOTCONV;
                cont = 0u;
            } else {
                o->beta = v[0] / o->rho;
                o->rho = v[0];
            }
        } else {
            o->cap = (o->iter >= o->max_iter);
            if (!(rel == rel)) {
                o->status = ST_BREAKDOWN;
                cont = 0u;
            }
        }
        if (!cont) {
            o->done = 1;
            o->skip_next = 1;
            set_cond(ctl, slot, 0u);
        } else {
            o->skip_next = 0;
        }
    }
}

// SIMPLE: z = S-hat^-1 r minus its component means; rho' = r.z, ||z||; preconditioned
// test; beta.
template <typename TX>
__global__ void k_outer_dots(Dev g, const int* __restrict__ cmp, const double* __restrict__ cmean,
                             const TX* __restrict__ sx, const double* __restrict__ rv,
                             Ctl* ctl, double* partials, int slot) {
    count_launch(ctl);
    CgState* o = &ctl->out;
    if (o->done) return;
    double v[2] = {0.0, 0.0};
    STREAM_LOOP(c, g.ncell) {
        const int k = cmp[c];
        const double zc = (k >= 0) ? (double)sx[c] - cmean[k] : 0.0;
        v[0] += rv[c] * zc;
        v[1] += zc * zc;
    }
    if (reduce_last_block<2>(v, partials, &ctl->ticket) && is_thread0()) {
        o->relz = sqrt(v[1] / o->zz0);
        unsigned cont = 1u;
        if (ctl->stop_norm == 1 && o->relz < o->tol) {
            o->status = ST_OK;
            cont = 0u;
        } else if (o->cap) {
            o->status = ST_NOTCONV;
            cont = 0u;
        } else {
            o->beta = v[0] / o->rho;
            o->rho = v[0];
        }
        if (!cont) {
            o->done = 1;
            set_cond(ctl, slot, 0u);
        }
    }
}

// d = z + beta d (Uzawa: z = r).  `gate` is out.done for PCG and out.skip_next for FCG.
template <typename TX>
__global__ void k_outer_dir(Dev g, const int* __restrict__ cmp, const double* __restrict__ cmean,
                            const TX* __restrict__ sx, const double* __restrict__ rv,
                            double* __restrict__ dv, Ctl* ctl, const int* gate) {
    count_launch(ctl);
    const CgState* o = &ctl->out;
    if (*gate) return;
    const double beta = o->beta;
    if (ctl->precond == 0) {
        STREAM_LOOP(c, g.ncell) dv[c] = rv[c] + beta * dv[c];
    } else {
        STREAM_LOOP(c, g.ncell) {
            const int k = cmp[c];
            const double zc = (k >= 0) ? (double)sx[c] - cmean[k] : 0.0;
            dv[c] = zc + beta * dv[c];
        }
    }
}

// ------------------------------------------------------------------------------------
// mixed precision: flexible CG steps inside FP64 defect correction
// ------------------------------------------------------------------------------------

// Start of a refinement step: d = z_0 (Uzawa: r), ||r||^2 of the step's true residual.
template <typename TX>
__global__ void k_fcg_start(Dev g, const int* __restrict__ cmp, const double* __restrict__ cmean,
                            const TX* __restrict__ sx, const double* __restrict__ rv,
                            double* __restrict__ dv, Ctl* ctl, double* partials, int slot) {
    count_launch(ctl);
    double v[1] = {0.0};
    const int simple = ctl->precond == 1;
    STREAM_LOOP(c, g.ncell) {
        double zc;
        if (simple) {
            const int k = cmp[c];
            zc = (k >= 0) ? (double)sx[c] - cmean[k] : 0.0;
        } else {
            zc = rv[c];
        }
        dv[c] = zc;
        v[0] += rv[c] * rv[c];
    }
    if (reduce_last_block<1>(v, partials, &ctl->ticket) && is_thread0()) {
        ctl->mix.rr_step0 = v[0];
        ctl->mix.step_iter = 0;
        ctl->out.skip_next = 0;
        set_cond(ctl, slot, v[0] > 0.0 ? 1u : 0u);
    }
}

// q = B u (u = A^-1 B^T d in T); alpha = d.r / d.q (flexible CG).
template <typename TX>
__global__ void k_fcg_div(Dev g, const uint8_t* __restrict__ mask, const uint8_t* __restrict__ flags,
                          const TX* __restrict__ u, const double* __restrict__ dv,
                          const double* __restrict__ rv, double* __restrict__ qv, Ctl* ctl,
                          double* partials, int slot, int slot_ref) {
    count_launch(ctl);
    double v[2] = {0.0, 0.0};
    TILE_LOOP_BEGIN(g)
        double qc = 0.0;
        if (mask[c] == 1) {
            double s = 0.0;
            for (int a = 0; a < g.d; ++a) {
                int ex, ey, ez;
                axis_step(a, 1, ex, ey, ez);
                s += face_val(g, flags, u, a, x + ex, y + ey, z + ez) - face_val(g, flags, u, a, x, y, z);
            }
            qc = -g.hinv * s;
            v[0] += dv[c] * qc;
            v[1] += dv[c] * rv[c];
        }
        qv[c] = qc;
    TILE_LOOP_END
    if (reduce_last_block<2>(v, partials, &ctl->ticket) && is_thread0()) {
        CgState* o = &ctl->out;
        const double dq = v[0];
        if (!(dq > 0.0) || isinf(dq)) {
            o->status = ST_BREAKDOWN;
            o->alpha = 0.0;
            o->skip_next = 1;
            ctl->mix.stop = 1;
            set_cond(ctl, slot, 0u);
            set_cond(ctl, slot_ref, 0u);
        } else {
            o->alpha = v[1] / dq;
            ctl->mix.dq = dq;
        }
    }
}

// p += alpha d, r -= alpha q; the step ends when ||r|| fell by `factor`, or the global
// tolerance is met on the recursive residual, or a cap is reached.
__global__ void k_fcg_update(Dev g, double* __restrict__ pv, double* __restrict__ rv,
                             const double* __restrict__ dv, const double* __restrict__ qv,
                             Ctl* ctl, double* partials, int slot) {
    count_launch(ctl);
    CgState* o = &ctl->out;
    if (o->skip_next) return;
    const double alpha = o->alpha;
    double v[1] = {0.0};
    STREAM_LOOP(c, g.ncell) {
        pv[c] += alpha * dv[c];
        const double r = rv[c] - alpha * qv[c];
        rv[c] = r;
        v[0] += r * r;
    }
    if (reduce_last_block<1>(v, partials, &ctl->ticket) && is_thread0()) {
        Mix& m = ctl->mix;
        o->iter += 1;
        o->total += 1;
        m.step_iter += 1;
        const double f2 = m.factor * m.factor;
        const int done = (v[0] <= f2 * m.rr_step0) || (v[0] < o->tol * o->tol * o->rr0) ||
                         (m.step_iter >= m.step_max) || (o->iter >= o->max_iter) ||
                         !(v[0] == v[0]);
        if (done) {
            o->skip_next = 1;
            set_cond(ctl, slot, 0u);
        }
    }
}

// FCG(1) direction coefficient: beta = -z.q / d.q (z with its component means removed).
template <typename TX>
__global__ void k_fcg_dots(Dev g, const int* __restrict__ cmp, const double* __restrict__ cmean,
                           const TX* __restrict__ sx, const double* __restrict__ rv,
                           const double* __restrict__ qv, Ctl* ctl, double* partials) {
    count_launch(ctl);
    CgState* o = &ctl->out;
    if (o->skip_next) return;
    const int simple = ctl->precond == 1;
    double v[1] = {0.0};
    STREAM_LOOP(c, g.ncell) {
        double zc;
        if (simple) {
            const int k = cmp[c];
            zc = (k >= 0) ? (double)sx[c] - cmean[k] : 0.0;
        } else {
            zc = rv[c];
        }
        v[0] += zc * qv[c];
    }
    if (reduce_last_block<1>(v, partials, &ctl->ticket) && is_thread0())
        o->beta = -v[0] / ctl->mix.dq;
}

// True residual r = g - B u with u = A^-1 B^T p from an FP64 inner solve; decides whether
// another refinement step follows.
__global__ void k_true_res(Dev g, const uint8_t* __restrict__ mask, const uint8_t* __restrict__ flags,
                           const double* __restrict__ u, const double* __restrict__ gv,
                           double* __restrict__ rv, Ctl* ctl, double* partials, int slot_ref) {
    count_launch(ctl);
    if (ctl->mix.stop) return;
    double v[1] = {0.0};
    TILE_LOOP_BEGIN(g)
        double rc = 0.0;
        if (mask[c] == 1) {
            double s = 0.0;
            for (int a = 0; a < g.d; ++a) {
                int ex, ey, ez;
                axis_step(a, 1, ex, ey, ez);
                s += face_val(g, flags, u, a, x + ex, y + ey, z + ez) - face_val(g, flags, u, a, x, y, z);
            }
            rc = gv[c] + g.hinv * s;  // g - B u with B u = -h^-1 sum
            v[0] += rc * rc;
        }
        rv[c] = rc;
    TILE_LOOP_END
    if (reduce_last_block<1>(v, partials, &ctl->ticket) && is_thread0()) {
        CgState* o = &ctl->out;
        Mix& m = ctl->mix;
        const double rel = sqrt(v[0] / o->rr0);
        o->rel = rel;
        m.refine += 1;
        unsigned cont = 1u;
        if (rel < o->tol) {
            o->status = ST_OK;
            cont = 0u;
        } else if (!(rel == rel)) {
            o->status = ST_BREAKDOWN;
            cont = 0u;
        } else if (m.refine >= m.max_refine || o->iter >= o->max_iter) {
            o->status = ST_NOTCONV;
            cont = 0u;
        }
        if (!cont) set_cond(ctl, slot_ref, 0u);
    }
}

// u = x (the recovered velocity) and the per-axis sums of u for the permeability.
__global__ void k_copy_u(Dev g, const uint8_t* __restrict__ flags, const double* __restrict__ xv,
                         double* __restrict__ u, Ctl* ctl, double* partials) {
    count_launch(ctl);
    double v[3] = {0.0, 0.0, 0.0};
    const long long n = (long long)g.d * g.stride;
    STREAM_LOOP(i, n) {
        const double xi = (flags[i] & 1) ? xv[i] : 0.0;
        u[i] = xi;
        const int a = (int)(i / g.stride);
        v[0] += (a == 0) ? xi : 0.0;
        v[1] += (a == 1) ? xi : 0.0;
        v[2] += (a == 2) ? xi : 0.0;
    }
    if (reduce_last_block<3>(v, partials, &ctl->ticket) && is_thread0()) {
        for (int a = 0; a < 3; ++a) ctl->perm[a] = v[a] / (double)g.ncell;
    }
}

// ------------------------------------------------------------------------------------
// recorded control flow
// ------------------------------------------------------------------------------------

static inline dim3 tblock() { return dim3(kTileX, kTileY, 1); }
static inline dim3 tgrid(const Handle& H) {
    const long long gx = (H.g.nx + kTileX - 1) / kTileX, gy = (H.g.ny + kTileY - 1) / kTileY;
    const long long nt = gx * gy * H.g.nz;
    return dim3((unsigned)(nt < H.target_blocks ? nt : H.target_blocks));
}
static inline dim3 sgrid(const Handle& H, long long n) {
    const long long nb = (n + kBlock - 1) / kBlock;
    return dim3((unsigned)(nb < H.target_blocks ? (nb > 0 ? nb : 1) : H.target_blocks));
}
static inline dim3 sblock() { return dim3(kBlock); }
// column-tile grid: x = strided x-y tiles, y = z chunks, z = fields
static inline dim3 cgrid(const Handle& H, int fields) {
    const long long tiles = (long long)((H.g.nx + kTileX - 1) / kTileX) * ((H.g.ny + kTileY - 1) / kTileY);
    const long long target = H.target_blocks;
    long long zs = 1, gxx = tiles;
    if (tiles * fields >= target) {
        gxx = (target + fields - 1) / fields;
    } else {
        zs = (target + tiles * fields - 1) / (tiles * fields);
        if (zs > H.g.nz) zs = H.g.nz;
    }
    if (gxx < 1) gxx = 1;
    return dim3((unsigned)gxx, (unsigned)zs, (unsigned)fields);
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
};
static InnerA<double> innerA64(Handle& H) { return {H.ax, H.ar, H.ap, H.aq}; }
static InnerA<float> innerA32(Handle& H) { return {H.axf, H.arf, H.apf, H.aqf}; }
static InnerS<double> innerS64(Handle& H) { return {H.sx, H.sr, H.sp, H.sq, H.invdS}; }
static InnerS<float> innerS32(Handle& H) { return {H.sxf, H.srf, H.spf, H.sqf, H.invdSf}; }

// x = A^-1 b with b = cf f + cp B^T P (+ bvec) formed by k_cgA_init.
template <typename T>
static void record_A_solve(Handle& H, Recorder& R, InnerA<T> v, CgState* st, int s,
                           const double* P, double cp, double cf, const double* bvec) {
    R.launch("cgA_init", k_cgA_init<T>, cgrid(H, H.g.d), tblock(), H.g, (const uint8_t*)H.flags,
             v.x, v.r, P, cp, cf, bvec, H.dctl, st, H.partials, s);
    const long long nu = H.n_u;
    R.loop(s, [&H, v, st, s, nu](Recorder& B) {
        B.launch("cgA_dir", k_cgA_dir<T>, sgrid(H, nu), sblock(), H.g, (const uint32_t*)H.ulist, nu,
                 (const uint8_t*)H.flags, (const T*)v.r, v.p, H.dctl, (const CgState*)st);
        B.launch("cgA_matvec", k_cgA_matvec<T>, sgrid(H, nu), sblock(), H.g, (const uint32_t*)H.ulist,
                 nu, (const uint8_t*)H.flags, (const T*)v.p, v.q, H.dctl, st, H.partials, s);
        B.launch("cgA_update", k_cgA_update<T>, sgrid(H, nu), sblock(), H.g, (const uint32_t*)H.ulist,
                 nu, (const uint8_t*)H.flags, v.x, v.r, (const T*)v.p, (const T*)v.q, H.dctl, st,
                 H.partials, s);
    });
}

template <typename T>
static void record_comp_means(Handle& H, Recorder& R, const T* v) {
    const CgState* outer = &H.dctl->out;
    R.launch("comp_big", k_comp_big<T>, sgrid(H, H.g.ncell), sblock(), H.g, (const int*)H.cmp, v,
             H.cmean, H.n_big, H.dctl, outer, H.partials);
    if (H.n_small > 0) {
        const long long nb = (H.n_small + 7) / 8;
        const dim3 grid((unsigned)(nb < H.target_blocks ? nb : H.target_blocks));
        R.launch("comp_small", k_comp_small<T>, grid, sblock(), (const int*)H.small_start,
                 (const int*)H.small_cells, v, H.cmean, H.n_big, H.n_small, H.dctl, outer);
    }
}

// z = S-hat^+ r: r (the FP64 outer residual) is projected onto the range (component
// means removed, in place), the inner CG runs in T, and the per-component means of the
// solution are left in cmean for the consumers to subtract.
template <typename T>
static void record_S_solve(Handle& H, Recorder& R, InnerS<T> v, CgState* st, int s) {
    record_comp_means<double>(H, R, H.orr);
    R.launch("cgS_init", k_cgS_init<T>, sgrid(H, H.g.ncell), sblock(), H.g, v.invd,
             (const int*)H.cmp, (const double*)H.cmean, H.orr, v.x, v.r, H.dctl, st,
             (const CgState*)&H.dctl->out, H.partials, s);
    const long long np = H.n_p;
    R.loop(s, [&H, v, st, s, np](Recorder& B) {
        B.launch("cgS_dir", k_cgS_dir<T>, sgrid(H, np), sblock(), H.g, (const uint32_t*)H.flist, np,
                 v.invd, (const T*)v.r, v.p, H.dctl, (const CgState*)st);
        B.launch("cgS_matvec", k_cgS_matvec<T>, sgrid(H, np), sblock(), H.g, (const uint32_t*)H.flist,
                 np, (const uint8_t*)H.flags, (const T*)v.p, v.q, H.dctl, st, H.partials, s);
        B.launch("cgS_update", k_cgS_update<T>, sgrid(H, np), sblock(), H.g, (const uint32_t*)H.flist,
                 np, v.invd, v.x, v.r, (const T*)v.p, (const T*)v.q, H.dctl, st, H.partials, s);
    });
    record_comp_means<T>(H, R, (const T*)v.x);
}

// Algorithm 1 in FP64.
static void record_solve_fp64(Handle& H, Recorder& R, int precond) {
    Ctl* ctl = H.dctl;
    CgState* inA = &ctl->inA;
    CgState* inS = &ctl->inS;
    const InnerA<double> A = innerA64(H);
    const InnerS<double> S = innerS64(H);
    // slots are allocated before any loop body is recorded: in host-driven mode a body
    // runs once per iteration and must not allocate
    const int s_rhs = R.new_slot();
    const int s_out = R.new_slot();
    const int s_s0 = R.new_slot();
    const int s_a = R.new_slot();
    const int s_s = R.new_slot();
    record_A_solve<double>(H, R, A, inA, s_rhs, nullptr, 0.0, 1.0, nullptr);   // A^-1 f
    R.launch("outer_init", k_outer_init<double>, tgrid(H), tblock(), H.g, (const uint8_t*)H.mask,
             (const uint8_t*)H.flags, (const double*)A.x, H.og, H.orr, H.op, H.od, ctl, H.partials,
             s_out);
    if (precond == 1) {
        record_S_solve<double>(H, R, S, inS, s_s0);
        R.launch("outer_start", k_outer_start<double>, sgrid(H, H.g.ncell), sblock(), H.g,
                 (const int*)H.cmp, (const double*)H.cmean, (const double*)S.x,
                 (const double*)H.orr, H.od, ctl, H.partials, s_out);
    }
    R.loop(s_out, [&H, ctl, inA, inS, A, S, precond, s_out, s_a, s_s](Recorder& B) {
        // q = S d = B A^-1 B^T d
        record_A_solve<double>(H, B, A, inA, s_a, H.od, 1.0, 0.0, nullptr);
        B.launch("outer_div", k_outer_div<double>, tgrid(H), tblock(), H.g, (const uint8_t*)H.mask,
                 (const uint8_t*)H.flags, (const double*)A.x, (const double*)H.od, H.oq, ctl,
                 H.partials, s_out);
        B.launch("outer_update", k_outer_update, sgrid(H, H.g.ncell), sblock(), H.g, H.op, H.orr,
                 (const double*)H.od, (const double*)H.oq, ctl, H.partials, s_out);
        if (precond == 1) {
            record_S_solve<double>(H, B, S, inS, s_s);
            B.launch("outer_dots", k_outer_dots<double>, sgrid(H, H.g.ncell), sblock(), H.g,
                     (const int*)H.cmp, (const double*)H.cmean, (const double*)S.x,
                     (const double*)H.orr, ctl, H.partials, s_out);
        }
        B.launch("outer_dir", k_outer_dir<double>, sgrid(H, H.g.ncell), sblock(), H.g,
                 (const int*)H.cmp, (const double*)H.cmean, (const double*)S.x, (const double*)H.orr,
                 H.od, ctl, (const int*)&ctl->out.done);
    });
}

// Mixed precision: FP64 defect correction around FP64 flexible CG with FP32 inner solves.
static void record_solve_mixed(Handle& H, Recorder& R, int precond) {
    Ctl* ctl = H.dctl;
    const InnerA<double> A64 = innerA64(H);
    const InnerA<float> A32 = innerA32(H);
    const InnerS<float> S32 = innerS32(H);
    CgState* inA = &ctl->inA;
    CgState* inA32 = &ctl->inA32;
    CgState* inS32 = &ctl->inS32;
    const int s_rhs = R.new_slot();
    const int s_ref = R.new_slot();
    const int s_s0 = R.new_slot();
    const int s_fcg = R.new_slot();
    const int s_a = R.new_slot();
    const int s_s = R.new_slot();
    const int s_t = R.new_slot();
    record_A_solve<double>(H, R, A64, inA, s_rhs, nullptr, 0.0, 1.0, nullptr);  // FP64 A^-1 f
    R.launch("outer_init", k_outer_init<double>, tgrid(H), tblock(), H.g, (const uint8_t*)H.mask,
             (const uint8_t*)H.flags, (const double*)A64.x, H.og, H.orr, H.op, H.od, ctl,
             H.partials, s_ref);
    R.loop(s_ref, [&H, ctl, A64, A32, S32, inA, inA32, inS32, precond, s_ref, s_s0, s_fcg, s_a,
                   s_s, s_t](Recorder& B) {
        if (precond == 1) record_S_solve<float>(H, B, S32, inS32, s_s0);
        B.launch("fcg_start", k_fcg_start<float>, sgrid(H, H.g.ncell), sblock(), H.g,
                 (const int*)H.cmp, (const double*)H.cmean, (const float*)S32.x,
                 (const double*)H.orr, H.od, ctl, H.partials, s_fcg);
        B.loop(s_fcg, [&H, ctl, A32, S32, inA32, inS32, precond, s_fcg, s_a, s_s,
                       s_ref](Recorder& C) {
            record_A_solve<float>(H, C, A32, inA32, s_a, H.od, 1.0, 0.0, nullptr);
            C.launch("fcg_div", k_fcg_div<float>, tgrid(H), tblock(), H.g, (const uint8_t*)H.mask,
                     (const uint8_t*)H.flags, (const float*)A32.x, (const double*)H.od,
                     (const double*)H.orr, H.oq, ctl, H.partials, s_fcg, s_ref);
            C.launch("fcg_update", k_fcg_update, sgrid(H, H.g.ncell), sblock(), H.g, H.op, H.orr,
                     (const double*)H.od, (const double*)H.oq, ctl, H.partials, s_fcg);
            if (precond == 1) record_S_solve<float>(H, C, S32, inS32, s_s);
            C.launch("fcg_dots", k_fcg_dots<float>, sgrid(H, H.g.ncell), sblock(), H.g,
                     (const int*)H.cmp, (const double*)H.cmean, (const float*)S32.x,
                     (const double*)H.orr, (const double*)H.oq, ctl, H.partials);
            C.launch("fcg_dir", k_outer_dir<float>, sgrid(H, H.g.ncell), sblock(), H.g,
                     (const int*)H.cmp, (const double*)H.cmean, (const float*)S32.x,
                     (const double*)H.orr, H.od, ctl, (const int*)&ctl->out.skip_next);
        });
        // true residual with an FP64 inner solve: r = g - B A^-1 B^T p
        record_A_solve<double>(H, B, A64, inA, s_t, H.op, 1.0, 0.0, nullptr);
        B.launch("true_res", k_true_res, tgrid(H), tblock(), H.g, (const uint8_t*)H.mask,
                 (const uint8_t*)H.flags, (const double*)A64.x, (const double*)H.og, H.orr, ctl,
                 H.partials, s_ref);
    });
}

void record_solve(Handle& H, Recorder& R, int precond, int precision) {
    if (precision == 1) record_solve_mixed(H, R, precond);
    else record_solve_fp64(H, R, precond);
}

void record_solve_recover(Handle& H, Recorder& R, int precond, int precision) {
    record_solve(H, R, precond, precision);
    record_recover(H, R);
}

void record_recover(Handle& H, Recorder& R) {
    Ctl* ctl = H.dctl;
    const int s = R.new_slot();
    record_A_solve<double>(H, R, innerA64(H), &ctl->rec, s, H.op, -1.0, 1.0, nullptr);
    const long long nf = (long long)H.g.d * H.g.stride;
    R.launch("copy_u", k_copy_u, sgrid(H, nf), sblock(), H.g, (const uint8_t*)H.flags,
             (const double*)H.ax, H.u, ctl, H.partials);
}

void record_solve_A(Handle& H, Recorder& R, const double* b, double* x) {
    const int s = R.new_slot();
    record_A_solve<double>(H, R, innerA64(H), &H.dctl->solo, s, nullptr, 0.0, 0.0, b);
    (void)x;
}

// One launch of a hot kernel on the handle's stream between two CUDA events (the
// kernels read and write the solver's own buffers; the solo CG state absorbs the
// scalars).  which: 0-5 FP64 A dir/matvec/update and S dir/matvec/update; 6-11 the same
// in FP32 (the mixed-precision buffers must exist).
cudaError_t time_kernel(Handle& H, int which, int slot, float* ms) {
    if (!H.ev0) {
        cudaError_t e = cudaEventCreate(&H.ev0);
        if (e == cudaSuccess) e = cudaEventCreate(&H.ev1);
        if (e != cudaSuccess) return e;
    }
    if (which >= 6 && !H.axf) return cudaErrorInvalidValue;
    Ctl* ctl = H.dctl;
    CgState* st = &ctl->solo;
    const long long nu = H.n_u, np = H.n_p;
    cudaError_t e = cudaEventRecord(H.ev0, H.stream);
    if (e != cudaSuccess) return e;
    const dim3 gu = sgrid(H, nu), gp = sgrid(H, np), b = sblock();
    cudaStream_t s = H.stream;
    switch (which) {
        case 0: k_cgA_dir<double><<<gu, b, 0, s>>>(H.g, H.ulist, nu, H.flags, H.ar, H.ap, ctl, st); break;
        case 1: k_cgA_matvec<double><<<gu, b, 0, s>>>(H.g, H.ulist, nu, H.flags, H.ap, H.aq, ctl, st, H.partials, slot); break;
        case 2: k_cgA_update<double><<<gu, b, 0, s>>>(H.g, H.ulist, nu, H.flags, H.ax, H.ar, H.ap, H.aq, ctl, st, H.partials, slot); break;
        case 3: k_cgS_dir<double><<<gp, b, 0, s>>>(H.g, H.flist, np, H.invdS, H.sr, H.sp, ctl, st); break;
        case 4: k_cgS_matvec<double><<<gp, b, 0, s>>>(H.g, H.flist, np, H.flags, H.sp, H.sq, ctl, st, H.partials, slot); break;
        case 5: k_cgS_update<double><<<gp, b, 0, s>>>(H.g, H.flist, np, H.invdS, H.sx, H.sr, H.sp, H.sq, ctl, st, H.partials, slot); break;
        case 6: k_cgA_dir<float><<<gu, b, 0, s>>>(H.g, H.ulist, nu, H.flags, H.arf, H.apf, ctl, st); break;
        case 7: k_cgA_matvec<float><<<gu, b, 0, s>>>(H.g, H.ulist, nu, H.flags, H.apf, H.aqf, ctl, st, H.partials, slot); break;
        case 8: k_cgA_update<float><<<gu, b, 0, s>>>(H.g, H.ulist, nu, H.flags, H.axf, H.arf, H.apf, H.aqf, ctl, st, H.partials, slot); break;
        case 9: k_cgS_dir<float><<<gp, b, 0, s>>>(H.g, H.flist, np, H.invdSf, H.srf, H.spf, ctl, st); break;
        case 10: k_cgS_matvec<float><<<gp, b, 0, s>>>(H.g, H.flist, np, H.flags, H.spf, H.sqf, ctl, st, H.partials, slot); break;
        case 11: k_cgS_update<float><<<gp, b, 0, s>>>(H.g, H.flist, np, H.invdSf, H.sxf, H.srf, H.spf, H.sqf, ctl, st, H.partials, slot); break;
        default: return cudaErrorInvalidValue;
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(H.ev1, H.stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(H.ev1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, H.ev0, H.ev1);
    return e;
}

}  // namespace schur
