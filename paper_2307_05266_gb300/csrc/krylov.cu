// Krylov kernels and the recorded control flow of a solve.
//
// Inner solves: Jacobi-preconditioned CG from x_0 = 0 with the stopping rule of
// Section 3.2, ||M^-1 r_k|| / ||M^-1 r_0|| < eps, for A (face space, M = diag(A)) and
// for S-hat_simple (cell space, M = diag(S-hat)).  One CG iteration has three phases:
//   dir:    p = z + beta p  (z = M^-1 r formed on the fly; beta = 0 on the first pass)
//   matvec: q = Op p and p.q, then alpha = rho / p.q
//   update: x += alpha p, r -= alpha q, r.z and z.z, then beta, the convergence test
// An init kernel forms the right-hand side and starts the state; then one persistent
// kernel, launched cooperatively so that its blocks are co-resident, runs every
// iteration with grid barriers between the phases (three per iteration), and every block
// sums the dot products of all blocks in the same fixed order, so that all blocks hold
// the same scalars and take the same decisions.  Each barrier wait is bounded; a wait
// that runs out sets a sticky error flag, and every kernel, loop and the host call then
// stop with an error status.  The phases also run as single kernels, one graph node each
// inside a conditional while node, in the per-phase launch shape (geometries that share
// the GPU interleave better that way) and in the profiling hook.
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
// Layout: the vectors of the inner solves are compact, one entry per unknown face (in
// (a, z, y, x) order) or per fluid cell (in (z, y, x) order), so the streaming phases
// are dense, coalesced loops; stencil neighbours come from per-geometry tables (built
// from per-row bitmaps: for every row of nx positions, one 32-bit word per 32 positions
// and the compact index of that word's first set bit, so a rank is base + popcount).  The
// outer vectors stay dense in cell space (0 on solid cells).
// All scalars live in the device control block; every outer loop is a conditional while
// node of one CUDA graph (or a host loop in debugging mode).  Every loop terminates: each
// condition update either continues below its iteration cap or stops.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>

#include "cg_dev.cuh"

namespace schur {



// Neighbour tables, one thread per entry: the rank lookups of the row bitmaps run once
// per geometry instead of once per stencil application.
__global__ void k_build_nbA(Dev g, Compact C, uint32_t* __restrict__ nbA) {
    STREAM_LOOP(k, C.n_u) {
        const FaceAt f = decode_face(g, C.ulist[k]);
        for (int e = 0; e < 2 * g.d; ++e) {
            const int b = e >> 1, sgn = (e & 1) ? 1 : -1;
            const long long r = face_rank(g, C, f.a, f.x + (b == 0) * sgn, f.y + (b == 1) * sgn,
                                          f.z + (b == 2) * sgn);
            nbA[e * C.ldA + k] = r < 0 ? (uint32_t)C.n_u : (uint32_t)r;
        }
    }
}

// Direction e = 2a is the lower face (a, c), e = 2a + 1 the upper face (a, c + e_a); an
// open (unknown) face links the cell to the fluid cell on its other side.  dS is the
// diagonal of S-hat_simple, the sum of the open faces' weights.
__global__ void k_build_nbS(Dev g, Compact C, const uint8_t* __restrict__ flags,
                            uint32_t* __restrict__ nbS, uint32_t* __restrict__ codeS,
                            double* __restrict__ dS) {
    STREAM_LOOP(m, C.n_p) {
        const FaceAt f = decode_face(g, C.flist[m]);
        uint32_t code = 0;
        double diag = 0.0;
        for (int e = 0; e < 2 * g.d; ++e) {
            const int a = e >> 1, up = e & 1;
            const int ex = a == 0, ey = a == 1, ez = a == 2;
            uint32_t nb = (uint32_t)C.n_p;
            int fx = f.x + up * ex, fy = f.y + up * ey, fz = f.z + up * ez;   // face position
            if (wrap3(g, fx, fy, fz)) {
                const uint8_t fl = flags[(long long)a * g.stride + ((long long)fz * g.ny + fy) * g.nx + fx];
                if (fl & 1) {
                    // the cell across the face: c - e_a (lower face) or c + e_a (upper face)
                    const long long r = up ? cell_rank(g, C, fx, fy, fz)
                                           : cell_rank(g, C, f.x - ex, f.y - ey, f.z - ez);
                    if (r >= 0) {
                        nb = (uint32_t)r;
                        const int gh = (fl >> 1) & 7;
                        code |= (uint32_t)(1 + gh) << (3 * e);
                        diag += tab5(g.wdiag, gh);
                    }
                }
            }
            nbS[e * C.ldS + m] = nb;
        }
        codeS[m] = code;
        dS[m] = diag;
    }
}

// ------------------------------------------------------------------------------------
// inner CG on A (compact face space)
// ------------------------------------------------------------------------------------
// The inner A solve works with the dimensionless operator A' = h^2 A (diagonal 2d + g,
// off-diagonal -1) and M' = diag(A'), right-hand side h^2 b: alpha, beta and every
// iterate x are those of CG on A x = b with Jacobi M = diag(A), without h^-2 factors.

// b = cf f_a + cp h^-1 (P_c - P_(c-e_a)) (+ bvec, dense face layout) on the unknowns
// (formed in FP64); x = 0, r = h^2 b.  P is a dense cell vector.
template <typename T>
__global__ void k_cgA_init(Dev g, Compact C, T* __restrict__ xv, T* __restrict__ rv,
                           const double* __restrict__ P, double cp, double cf,
                           const double* __restrict__ bvec, Ctl* ctl, CgState* st,
                           double* partials, int slot) {
    count_launch(ctl);
    double v[2] = {0.0, 0.0};
    const long long plane = (long long)g.nx * g.ny;
    STREAM_LOOP(k, C.n_u) {
        const uint32_t i = C.ulist[k];
        const FaceAt f = decode_face(g, i);
        const int a = f.a;
        double b = cf * ctl->f[a];
        if (P) {
            // an unknown face has a fluid lower cell inside the box (wrap when periodic)
            long long cl;
            if (a == 0) cl = f.x > 0 ? f.c - 1 : f.c + g.nx - 1;
            else if (a == 1) cl = f.y > 0 ? f.c - g.nx : f.c + (long long)(g.ny - 1) * g.nx;
            else cl = f.z > 0 ? f.c - plane : f.c + (long long)(g.nz - 1) * plane;
            b += cp * (g.hinv * (P[f.c] - P[cl]));
        }
        if (bvec) b += bvec[i];
        const T bt = (T)(b * g.h2);  // right-hand side of h^2 A x = h^2 b
        const double bd = (double)bt;
        const double zz = bd * tab5(g.wdiag, C.ufl[k] >> 1);
        v[0] += bd * zz;
        v[1] += zz * zz;
        xv[k] = (T)0;
        rv[k] = bt;
    }
    if (reduce_last_block<2>(v, partials, &ctl->ticket) && is_thread0()) {
        const unsigned go = start_inner(ctl, st, v[0], v[1]);
        ctl->bar_count = 0u;  // the loop kernel's grid barrier starts from zero arrivals
        if (slot >= 0) set_cond(ctl, slot, go);
    }
}


// The three phases of one inner CG iteration on A', as device functions shared by the
// single-phase kernels and the persistent loop kernel.  dir and update map entries to
// threads identically, so a thread only ever touches its own entries between barriers.

// p = M'^-1 r + beta p.
template <typename T>
__device__ __forceinline__ void phaseA_dir(const Tabs<T>& t, uint32_t n, const uint8_t* __restrict__ ufl,
                                           const T* __restrict__ rv, T* __restrict__ pv, T beta) {
    constexpr int kU = StreamU<T>::v;
    WARP_STREAM_BEGIN_U(n, kU)
        int gh[kU];
        T r[kU], p[kU];
#pragma unroll
        for (int j = 0; j < kU; ++j)
            if (idx[j] < n) { gh[j] = ufl[idx[j]] >> 1; r[j] = rv[idx[j]]; p[j] = pv[idx[j]]; }
#pragma unroll
        for (int j = 0; j < kU; ++j)
            if (idx[j] < n) pv[idx[j]] = r[j] * t.w[1 + gh[j]] + beta * p[j];
    WARP_STREAM_END
}


// x += alpha p, r -= alpha q; adds this thread's parts of r.z and z.z (z = M'^-1 r).
template <typename T>
__device__ __forceinline__ void phaseA_update(const Tabs<T>& t, uint32_t n, const uint8_t* __restrict__ ufl,
                                              T* __restrict__ xv, T* __restrict__ rv,
                                              const T* __restrict__ pv, const T* __restrict__ qv,
                                              T alpha, T& a0, T& a1) {
    constexpr int kU = StreamU<T>::v;
    WARP_STREAM_BEGIN_U(n, kU)
        int gh[kU];
        T xx[kU], p[kU], r[kU], q[kU];
#pragma unroll
        for (int j = 0; j < kU; ++j)
            if (idx[j] < n) {
                gh[j] = ufl[idx[j]] >> 1;
                xx[j] = xv[idx[j]];
                p[j] = pv[idx[j]];
                r[j] = rv[idx[j]];
                q[j] = qv[idx[j]];
            }
#pragma unroll
        for (int j = 0; j < kU; ++j)
            if (idx[j] < n) {
                xv[idx[j]] = xx[j] + alpha * p[j];
                const T rn = r[j] - alpha * q[j];
                rv[idx[j]] = rn;
                const T zz = rn * t.w[1 + gh[j]];
                a0 += rn * zz;
                a1 += zz * zz;
            }
    WARP_STREAM_END
}

// Single-phase kernels (one launch per phase; the profiling hook times them one by one).
template <typename T>
__global__ void k_cgA_dir(Dev g, long long n, const uint8_t* __restrict__ ufl,
                          const T* __restrict__ rv, T* __restrict__ pv, Ctl* ctl,
                          const CgState* st) {
    count_launch(ctl);
    __shared__ Tabs<T> t;
    load_tabs<T>(g, t);
    phaseA_dir<T>(t, (uint32_t)n, ufl, rv, pv, (T)(st->first ? 0.0 : st->beta));
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_cgA_matvec(Dev g, Compact C, const T* __restrict__ pv,
                                                       T* __restrict__ qv, Ctl* ctl, CgState* st,
                                                       double* partials, int slot) {
    count_launch(ctl);
    __shared__ Tabs<T> t;
    load_tabs<T>(g, t);
    double v[1] = {(double)phaseA_matvec<T>(t, g, C, pv, qv)};
    if (reduce_last_block<1>(v, partials, &ctl->ticket) && is_thread0())
        finish_matvec(ctl, st, v[0], slot);
}

template <typename T>
__global__ void k_cgA_update(Dev g, long long n, const uint8_t* __restrict__ ufl,
                             T* __restrict__ xv, T* __restrict__ rv, const T* __restrict__ pv,
                             const T* __restrict__ qv, Ctl* ctl, CgState* st,
                             double* partials, int slot) {
    count_launch(ctl);
    __shared__ Tabs<T> t;
    load_tabs<T>(g, t);
    T a0 = (T)0, a1 = (T)0;
    phaseA_update<T>(t, (uint32_t)n, ufl, xv, rv, pv, qv, (T)st->alpha, a0, a1);
    double v[2] = {(double)a0, (double)a1};
    if (reduce_last_block<2>(v, partials, &ctl->ticket) && is_thread0())
        set_cond(ctl, slot, finish_inner(ctl, st, v[0], v[1]));
}

// ------------------------------------------------------------------------------------
// inner CG on S-hat_simple (compact cell space); M^-1 = invd (0 on isolated cells)
// ------------------------------------------------------------------------------------

// b = r - (its mean on r's fluid component): the dense FP64 outer residual r is projected
// onto the range of S-hat in place, then x = 0 and the CG residual starts at b.
template <typename T>
__global__ void k_cgS_init(Dev g, Compact C, const T* __restrict__ invd, const int* __restrict__ cmpc,
                           const double* __restrict__ cmean, double* __restrict__ b,
                           T* __restrict__ xv, T* __restrict__ rv, Ctl* ctl, CgState* st,
                           const CgState* outer, double* partials, int slot) {
    count_launch(ctl);
    if (outer->skip_next) {
        if (blockIdx.x == 0 && is_thread0() && slot >= 0) set_cond(ctl, slot, 0u);
        return;
    }
    double v[2] = {0.0, 0.0};
    STREAM_LOOP(m, C.n_p) {
        const uint32_t c = C.flist[m];
        const double bc = b[c] - cmean[cmpc[m]];
        b[c] = bc;
        const T bt = (T)bc;
        const double zz = (double)bt * (double)invd[m];
        v[0] += (double)bt * zz;
        v[1] += zz * zz;
        xv[m] = (T)0;
        rv[m] = bt;
    }
    if (reduce_last_block<2>(v, partials, &ctl->ticket) && is_thread0()) {
        const unsigned go = start_inner(ctl, st, v[0], v[1]);
        ctl->bar_count = 0u;  // the loop kernel's grid barrier starts from zero arrivals
        if (slot >= 0) set_cond(ctl, slot, go);
    }
}

template <typename T>
__device__ __forceinline__ void phaseS_dir(uint32_t n, const T* __restrict__ invd,
                                           const T* __restrict__ rv, T* __restrict__ pv, T beta) {
    constexpr int kU = StreamU<T>::v;
    WARP_STREAM_BEGIN_U(n, kU)
        T r[kU], w[kU], p[kU];
#pragma unroll
        for (int j = 0; j < kU; ++j)
            if (idx[j] < n) { r[j] = rv[idx[j]]; w[j] = invd[idx[j]]; p[j] = pv[idx[j]]; }
#pragma unroll
        for (int j = 0; j < kU; ++j)
            if (idx[j] < n) pv[idx[j]] = r[j] * w[j] + beta * p[j];
    WARP_STREAM_END
}


template <typename T>
__device__ __forceinline__ void phaseS_update(uint32_t n, const T* __restrict__ invd, T* __restrict__ xv,
                                              T* __restrict__ rv, const T* __restrict__ pv,
                                              const T* __restrict__ qv, T alpha, T& a0, T& a1) {
    constexpr int kU = StreamU<T>::v;
    WARP_STREAM_BEGIN_U(n, kU)
        T xx[kU], p[kU], r[kU], q[kU], w[kU];
#pragma unroll
        for (int j = 0; j < kU; ++j)
            if (idx[j] < n) {
                xx[j] = xv[idx[j]];
                p[j] = pv[idx[j]];
                r[j] = rv[idx[j]];
                q[j] = qv[idx[j]];
                w[j] = invd[idx[j]];
            }
#pragma unroll
        for (int j = 0; j < kU; ++j)
            if (idx[j] < n) {
                xv[idx[j]] = xx[j] + alpha * p[j];
                const T rn = r[j] - alpha * q[j];
                rv[idx[j]] = rn;
                const T zz = rn * w[j];
                a0 += rn * zz;
                a1 += zz * zz;
            }
    WARP_STREAM_END
}

template <typename T>
__global__ void k_cgS_dir(Dev g, long long n, const T* __restrict__ invd, const T* __restrict__ rv,
                          T* __restrict__ pv, Ctl* ctl, const CgState* st) {
    count_launch(ctl);
    phaseS_dir<T>((uint32_t)n, invd, rv, pv, (T)(st->first ? 0.0 : st->beta));
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_cgS_matvec(Dev g, Compact C, const T* __restrict__ dS,
                                                       const T* __restrict__ pv, T* __restrict__ qv,
                                                       Ctl* ctl, CgState* st, double* partials,
                                                       int slot) {
    count_launch(ctl);
    __shared__ Tabs<T> t;
    load_tabs<T>(g, t);
    double v[1] = {(double)phaseS_matvec<T>(t, g, C, dS, pv, qv)};
    if (reduce_last_block<1>(v, partials, &ctl->ticket) && is_thread0())
        finish_matvec(ctl, st, v[0], slot);
}

template <typename T>
__global__ void k_cgS_update(Dev g, long long n, const T* __restrict__ invd, T* __restrict__ xv,
                             T* __restrict__ rv, const T* __restrict__ pv,
                             const T* __restrict__ qv, Ctl* ctl, CgState* st,
                             double* partials, int slot) {
    count_launch(ctl);
    T a0 = (T)0, a1 = (T)0;
    phaseS_update<T>((uint32_t)n, invd, xv, rv, pv, qv, (T)st->alpha, a0, a1);
    double v[2] = {(double)a0, (double)a1};
    if (reduce_last_block<2>(v, partials, &ctl->ticket) && is_thread0())
        set_cond(ctl, slot, finish_inner(ctl, st, v[0], v[1]));
}

// ------------------------------------------------------------------------------------
// persistent inner CG: one cooperative launch runs every iteration of an inner solve
// ------------------------------------------------------------------------------------
// The grid stays resident (one wave: the grid never exceeds the kernel's resident
// blocks), the phases are separated by grid barriers, and the dot products are summed
// by every block in the same fixed order, so all blocks hold bitwise-equal Krylov scalars
// and take the same decisions without writing them back between phases.  Three barriers
// per iteration replace three kernel launches and a conditional graph node.


// The loop of an inner solve after its init kernel: `st` holds the started state (status
// NOTCONV when iterations are due).  `gate` (may be null) skips the whole solve when set.
// Ends with st written back by block 0 and ctl->inner_status updated as the single-phase
// kernels do; a failed barrier leaves status ST_BARRIER.
template <typename T, bool kS>
__device__ __forceinline__ void cg_loop(const Dev& g, const Compact& C, const T* __restrict__ aux,
                                        const T* __restrict__ dS, T* __restrict__ xv, T* __restrict__ rv, T* __restrict__ pv,
                                        T* __restrict__ qv, Ctl* ctl, CgState* st, double* partials,
                                        const int* gate) {
    __shared__ CgState s;
    __shared__ unsigned s_cont;
    __shared__ Tabs<T> t;
    if (gate && *gate) return;
    load_tabs<T>(g, t);
    if (threadIdx.x == 0) s = *st;
    __syncthreads();
    if (s.status != ST_NOTCONV || ld_acquire_u32(&ctl->bar_err) != 0u) return;
    const uint32_t n = (uint32_t)(kS ? C.n_p : C.n_u);
    double* P1 = partials;               // [grid] p.q
    double* P2 = partials + kMaxBlocks;  // [grid][2] r.z, z.z
    unsigned target = 0;
    bool ok = true;
    for (;;) {
        const T beta = (T)(s.first ? 0.0 : s.beta);
        if constexpr (kS) phaseS_dir<T>(opaque_u32(n), opaque(aux), opaque(rv), opaque(pv), beta);
        else phaseA_dir<T>(t, opaque_u32(n), opaque(C.ufl), opaque(rv), opaque(pv), beta);
        if (!(ok = grid_barrier(ctl, target))) break;
        double v1[1];
        {
            Compact Cl = C;
            Cl.nbA = opaque(C.nbA);
            Cl.nbS = opaque(C.nbS);
            Cl.codeS = opaque(C.codeS);
            Cl.ufl = opaque(C.ufl);
            constexpr int U = LoopMvU<T>::v;
            if constexpr (kS)
                v1[0] = (double)phaseS_matvec<T, U>(t, g, Cl, opaque(dS), opaque(pv), opaque(qv));
            else
                v1[0] = (double)phaseA_matvec<T, U>(t, g, Cl, opaque(pv), opaque(qv));
        }
        if (!(ok = grid_sum<1>(v1, P1, ctl, target))) break;
        if (threadIdx.x == 0) {
            s_cont = matvec_alpha(&s, v1[0]) ? 1u : 0u;
            if (!s_cont) finish_inner(nullptr, &s, 0.0, 0.0);  // counts the iteration
        }
        __syncthreads();
        if (!s_cont) break;
        T a0 = (T)0, a1 = (T)0;
        if constexpr (kS)
            phaseS_update<T>(opaque_u32(n), opaque(aux), opaque(xv), opaque(rv), opaque(pv),
                             opaque(qv), (T)s.alpha, a0, a1);
        else
            phaseA_update<T>(t, opaque_u32(n), opaque(C.ufl), opaque(xv), opaque(rv), opaque(pv),
                             opaque(qv), (T)s.alpha, a0, a1);
        double v2[2] = {(double)a0, (double)a1};
        if (!(ok = grid_sum<2>(v2, P2, ctl, target))) break;
        if (threadIdx.x == 0) s_cont = finish_inner(nullptr, &s, v2[0], v2[1]);
        __syncthreads();
        if (!s_cont) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (!ok) s.status = ST_BARRIER;
        *st = s;
        note_inner_status(ctl, s.status);
    }
}

// Minimum resident blocks per SM asked of the loop kernels (3: the fused phases fit in 85
// registers without spills; the stencil phase of the loop kernel gathers 2 entries per
// thread and step in both precisions for that).
template <typename T> struct LoopMinBlocks { static constexpr int v = 3; };

// aux: unused for A; invd (Jacobi weights of S-hat) for S.  dS: diagonal of S-hat (read by
// the FP64 S matvec).
template <typename T>
__global__ void __launch_bounds__(kBlock, LoopMinBlocks<T>::v) k_cgA_loop(Dev g, Compact C, T* __restrict__ xv,
                                                     T* __restrict__ rv, T* __restrict__ pv,
                                                     T* __restrict__ qv, Ctl* ctl, CgState* st,
                                                     double* partials) {
    count_launch(ctl);
    cg_loop<T, false>(g, C, nullptr, nullptr, xv, rv, pv, qv, ctl, st, partials, nullptr);
}

template <typename T>
__global__ void __launch_bounds__(kBlock, LoopMinBlocks<T>::v) k_cgS_loop(Dev g, Compact C, const T* __restrict__ invd,
                                                     const T* __restrict__ dS, T* __restrict__ xv,
                                                     T* __restrict__ rv, T* __restrict__ pv,
                                                     T* __restrict__ qv, Ctl* ctl, CgState* st,
                                                     double* partials, const int* gate) {
    count_launch(ctl);
    cg_loop<T, true>(g, C, invd, dS, xv, rv, pv, qv, ctl, st, partials, gate);
}

// ------------------------------------------------------------------------------------
// per-component means (nullspace of S-hat_simple and S: constants per fluid component)
// ------------------------------------------------------------------------------------
// v is a dense cell vector (dense != 0: value at flist[m]) or a compact one (value at m).

// Means of v over the (at most kMaxBig) big components, summed by the whole grid.
template <typename T>
__global__ void k_comp_big(Dev g, Compact C, const int* __restrict__ cmpc, const T* __restrict__ v,
                           int dense, double* __restrict__ cmean, int nbig, Ctl* ctl,
                           const CgState* outer, double* partials) {
    count_launch(ctl);
    if (outer->skip_next) return;
    double s[kMaxBig];
#pragma unroll
    for (int b = 0; b < kMaxBig; ++b) s[b] = 0.0;
    STREAM_LOOP(m, C.n_p) {
        const int k = cmpc[m];
        if (k < nbig) {
            const double vc = (double)(dense ? v[C.flist[m]] : v[m]);
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
__global__ void k_comp_small(Compact C, const int* __restrict__ start, const int* __restrict__ cells,
                             const T* __restrict__ v, int dense, double* __restrict__ cmean,
                             int nbig, int nsmall, Ctl* ctl, const CgState* outer) {
    count_launch(ctl);
    if (outer->skip_next) return;
    const int lane = threadIdx.x & 31;
    const int warps = blockDim.x >> 5;
    for (long long j = (long long)blockIdx.x * warps + (threadIdx.x >> 5); j < nsmall;
         j += (long long)gridDim.x * warps) {
        const int b0 = start[j], b1 = start[j + 1];
        double s = 0.0;
        for (int i = b0 + lane; i < b1; i += 32) {
            const int m = cells[i];
            s += (double)(dense ? v[C.flist[m]] : v[m]);
        }
        s = warp_sum(s);
        if (lane == 0) cmean[nbig + j] = s / (double)(b1 - b0);
    }
}

// B u = -h^-1 sum_a (u_(a, c+e_a) - u_(a, c)) at fluid cell (x, y, z) from a compact face
// vector, and the sum of the magnitudes of its terms.
template <typename TX>
__device__ __forceinline__ double div_at(const Dev& g, const Compact& C, const TX* __restrict__ u,
                                         int x, int y, int z, double* mag) {
    double s = 0.0, sa = 0.0;
    for (int a = 0; a < g.d; ++a) {
        const double up = face_valc(g, C, u, a, x + (a == 0), y + (a == 1), z + (a == 2));
        const double lo = face_valc(g, C, u, a, x, y, z);
        s += up - lo;
        sa += fabs(up) + fabs(lo);
    }
    if (mag) *mag = g.hinv * sa;
    return -g.hinv * s;
}

// ------------------------------------------------------------------------------------
// outer Schur CG (Algorithm 1), dense cell space, FP64
// ------------------------------------------------------------------------------------

// g = B u (u = A^-1 f); r = g, p = 0, d = g; zero-RHS test.
template <typename TX>
__global__ void k_outer_init(Dev g, Compact C, const uint8_t* __restrict__ mask,
                             const TX* __restrict__ u, double* __restrict__ gv,
                             double* __restrict__ rv, double* __restrict__ pv,
                             double* __restrict__ dv, Ctl* ctl, double* partials, int slot) {
    count_launch(ctl);
    double v[2] = {0.0, 0.0};
    TILE_LOOP_BEGIN(g)
        double gc = 0.0;
        if (mask[c] == 1) {
            double mag;
            gc = div_at(g, C, u, x, y, z, &mag);
            v[0] += gc * gc;
            v[1] += mag * mag;
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
__global__ void k_outer_start(Dev g, Compact C, const int* __restrict__ cmpc,
                              const double* __restrict__ cmean, const TX* __restrict__ sx,
                              const double* __restrict__ rv, double* __restrict__ dv, Ctl* ctl,
                              double* partials, int slot) {
    count_launch(ctl);
    if (ctl->out.done) return;
    double v[2] = {0.0, 0.0};
    STREAM_LOOP(m, C.n_p) {
        const uint32_t c = C.flist[m];
        const double zc = (double)sx[m] - cmean[cmpc[m]];
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
__global__ void k_outer_div(Dev g, Compact C, const uint8_t* __restrict__ mask,
                            const TX* __restrict__ u, const double* __restrict__ dv,
                            double* __restrict__ qv, Ctl* ctl, double* partials, int slot) {
    count_launch(ctl);
    double v[1] = {0.0};
    TILE_LOOP_BEGIN(g)
        double qc = 0.0;
        if (mask[c] == 1) {
            qc = div_at(g, C, u, x, y, z, nullptr);
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
            hist_put(ctl, o->iter, H_ALPHA, o->alpha);
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
        hist_put(ctl, o->iter - 1, H_REL, rel);
        unsigned cont = 1u;
        if (ctl->bar_err) {
            o->status = ST_BARRIER;  // an inner solve failed: stop
            cont = 0u;
        } else if (ctl->stop_norm == 0 && rel < o->tol) {
            o->status = ST_OK;
            o->relz = nan("");
            cont = 0u;
        } else if (ctl->precond == 0) {
            // Uzawa: z = r
            o->relz = sqrt(v[0] / o->zz0);
            hist_put(ctl, o->iter - 1, H_RELZ, o->relz);
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
                hist_put(ctl, o->iter - 1, H_BETA, o->beta);
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
__global__ void k_outer_dots(Dev g, Compact C, const int* __restrict__ cmpc,
                             const double* __restrict__ cmean, const TX* __restrict__ sx,
                             const double* __restrict__ rv, Ctl* ctl, double* partials, int slot) {
    count_launch(ctl);
    CgState* o = &ctl->out;
    if (o->done) return;
    double v[2] = {0.0, 0.0};
    STREAM_LOOP(m, C.n_p) {
        const double zc = (double)sx[m] - cmean[cmpc[m]];
        v[0] += rv[C.flist[m]] * zc;
        v[1] += zc * zc;
    }
    if (reduce_last_block<2>(v, partials, &ctl->ticket) && is_thread0()) {
        o->relz = sqrt(v[1] / o->zz0);
        hist_put(ctl, o->iter - 1, H_RELZ, o->relz);
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
            hist_put(ctl, o->iter - 1, H_BETA, o->beta);
        }
        if (!cont) {
            o->done = 1;
            set_cond(ctl, slot, 0u);
        }
    }
}

// d = z + beta d (Uzawa: z = r).  `gate` is out.done for PCG and out.skip_next for FCG.
template <typename TX>
__global__ void k_outer_dir(Dev g, Compact C, const int* __restrict__ cmpc,
                            const double* __restrict__ cmean, const TX* __restrict__ sx,
                            const double* __restrict__ rv, double* __restrict__ dv, Ctl* ctl,
                            const int* gate) {
    count_launch(ctl);
    const CgState* o = &ctl->out;
    if (*gate) return;
    const double beta = o->beta;
    if (ctl->precond == 0) {
        STREAM_LOOP(c, g.ncell) dv[c] = rv[c] + beta * dv[c];
    } else {
        STREAM_LOOP(m, C.n_p) {
            const uint32_t c = C.flist[m];
            const double zc = (double)sx[m] - cmean[cmpc[m]];
            dv[c] = zc + beta * dv[c];
        }
    }
}

// ------------------------------------------------------------------------------------
// mixed precision: flexible CG steps inside FP64 defect correction
// ------------------------------------------------------------------------------------

// Start of a refinement step: d = z_0 (Uzawa: r), ||r||^2 of the step's true residual.
template <typename TX>
__global__ void k_fcg_start(Dev g, Compact C, const int* __restrict__ cmpc,
                            const double* __restrict__ cmean, const TX* __restrict__ sx,
                            const double* __restrict__ rv, double* __restrict__ dv, Ctl* ctl,
                            double* partials, int slot) {
    count_launch(ctl);
    double v[1] = {0.0};
    const int simple = ctl->precond == 1;
    STREAM_LOOP(m, C.n_p) {
        const uint32_t c = C.flist[m];
        const double rc = rv[c];
        dv[c] = simple ? (double)sx[m] - cmean[cmpc[m]] : rc;
        v[0] += rc * rc;
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
__global__ void k_fcg_div(Dev g, Compact C, const uint8_t* __restrict__ mask,
                          const TX* __restrict__ u, const double* __restrict__ dv,
                          const double* __restrict__ rv, double* __restrict__ qv, Ctl* ctl,
                          double* partials, int slot, int slot_ref) {
    count_launch(ctl);
    double v[2] = {0.0, 0.0};
    TILE_LOOP_BEGIN(g)
        double qc = 0.0;
        if (mask[c] == 1) {
            qc = div_at(g, C, u, x, y, z, nullptr);
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
            hist_put(ctl, o->iter, H_ALPHA, o->alpha);
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
        hist_put(ctl, o->iter - 1, H_REL, sqrt(v[0] / o->rr0));
        const double f2 = m.factor * m.factor;
        const int done = (v[0] <= f2 * m.rr_step0) || (v[0] < o->tol * o->tol * o->rr0) ||
                         (m.step_iter >= m.step_max) || (o->iter >= o->max_iter) ||
                         !(v[0] == v[0]) || ctl->bar_err;
        if (done) {
            o->skip_next = 1;
            set_cond(ctl, slot, 0u);
        }
    }
}

// FCG(1) direction coefficient: beta = -z.q / d.q (z with its component means removed).
template <typename TX>
__global__ void k_fcg_dots(Dev g, Compact C, const int* __restrict__ cmpc,
                           const double* __restrict__ cmean, const TX* __restrict__ sx,
                           const double* __restrict__ rv, const double* __restrict__ qv,
                           Ctl* ctl, double* partials) {
    count_launch(ctl);
    CgState* o = &ctl->out;
    if (o->skip_next) return;
    const int simple = ctl->precond == 1;
    double v[1] = {0.0};
    STREAM_LOOP(m, C.n_p) {
        const uint32_t c = C.flist[m];
        const double zc = simple ? (double)sx[m] - cmean[cmpc[m]] : rv[c];
        v[0] += zc * qv[c];
    }
    if (reduce_last_block<1>(v, partials, &ctl->ticket) && is_thread0()) {
        o->beta = -v[0] / ctl->mix.dq;
        hist_put(ctl, o->iter - 1, H_BETA, o->beta);
    }
}

// True residual r = g - B u with u = A^-1 B^T p from an FP64 inner solve; decides whether
// another refinement step follows.
__global__ void k_true_res(Dev g, Compact C, const uint8_t* __restrict__ mask,
                           const double* __restrict__ u, const double* __restrict__ gv,
                           double* __restrict__ rv, Ctl* ctl, double* partials, int slot_ref) {
    count_launch(ctl);
    if (ctl->mix.stop) return;
    double v[1] = {0.0};
    TILE_LOOP_BEGIN(g)
        double rc = 0.0;
        if (mask[c] == 1) {
            rc = gv[c] - div_at(g, C, u, x, y, z, nullptr);
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
        if (ctl->bar_err) {
            o->status = ST_BARRIER;
            cont = 0u;
        } else if (rel < o->tol) {
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

// u = x scattered to the dense face layout, and the per-axis sums for the permeability.
__global__ void k_copy_u(Dev g, Compact C, const double* __restrict__ xv, double* __restrict__ u,
                         Ctl* ctl, double* partials) {
    count_launch(ctl);
    double v[3] = {0.0, 0.0, 0.0};
    const uint32_t s = (uint32_t)g.stride;
    STREAM_LOOP(k, C.n_u) {
        const uint32_t i = C.ulist[k];
        const double xi = xv[k];
        u[i] = xi;
        const int a = (i >= s) + (i >= 2u * s);
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


// x = A^-1 b with b = cf f + cp B^T P (+ bvec) formed by k_cgA_init.
template <typename T>
static void record_A_solve(Handle& H, Recorder& R, InnerA<T> v, CgState* st, int s,
                           const double* P, double cp, double cf, const double* bvec) {
    const Compact C = compact_of(H);
    const long long nu = H.n_u;
    const bool mg = H.inner_precond == SCHUR_INNER_MG;
    if (H.persistent || mg) {
        R.launch("cgA_init", k_cgA_init<T>, sgrid(H, nu, k_cgA_init<T>), sblock(), H.g, C, v.x, v.r,
                 P, cp, cf, bvec, H.dctl, st, H.partials, -1);
        if (mg)
            record_mg_loop(H, R, false, sizeof(T) == sizeof(float), v.x, v.r, v.p, v.q, st, nullptr);
        else
            R.launch_coop("cgA_loop", k_cgA_loop<T>, lgrid(H, nu, k_cgA_loop<T>), sblock(), H.g, C,
                          v.x, v.r, v.p, v.q, H.dctl, st, H.partials);
        return;
    }
    // one graph node per phase inside a conditional while node: many geometries that share
    // the GPU interleave at phase granularity
    R.launch("cgA_init", k_cgA_init<T>, sgrid(H, nu, k_cgA_init<T>), sblock(), H.g, C, v.x, v.r, P,
             cp, cf, bvec, H.dctl, st, H.partials, s);
    R.loop(s, [&H, C, v, st, s, nu](Recorder& B) {
        B.launch("cgA_dir", k_cgA_dir<T>, sgrid(H, nu, k_cgA_dir<T>), sblock(), H.g, nu,
                 (const uint8_t*)H.ufl, (const T*)v.r, v.p, H.dctl, (const CgState*)st);
        B.launch("cgA_matvec", k_cgA_matvec<T>, sgrid(H, nu, k_cgA_matvec<T>), sblock(), H.g, C,
                 (const T*)v.p, v.q, H.dctl, st, H.partials, s);
        B.launch("cgA_update", k_cgA_update<T>, sgrid(H, nu, k_cgA_update<T>), sblock(), H.g, nu,
                 (const uint8_t*)H.ufl, v.x, v.r, (const T*)v.p, (const T*)v.q, H.dctl, st,
                 H.partials, s);
    });
}

template <typename T>
static void record_comp_means(Handle& H, Recorder& R, const T* v, int dense) {
    const CgState* outer = &H.dctl->out;
    const Compact C = compact_of(H);
    R.launch("comp_big", k_comp_big<T>, sgrid(H, H.n_p, k_comp_big<T>), sblock(), H.g, C, (const int*)H.cmpc, v,
             dense, H.cmean, H.n_big, H.dctl, outer, H.partials);
    if (H.n_small > 0) {
        const long long nb = (H.n_small + 7) / 8;
        const dim3 grid((unsigned)(nb < H.target_blocks ? nb : H.target_blocks));
        R.launch("comp_small", k_comp_small<T>, grid, sblock(), C, (const int*)H.small_start,
                 (const int*)H.small_cells, v, dense, H.cmean, H.n_big, H.n_small, H.dctl, outer);
    }
}

// z = S-hat^+ r: r (the dense FP64 outer residual) is projected onto the range (component
// means removed, in place), the inner CG runs in T on compact vectors, and the
// per-component means of the solution are left in cmean for the consumers to subtract.
template <typename T>
static void record_S_solve(Handle& H, Recorder& R, InnerS<T> v, CgState* st, int s) {
    const Compact C = compact_of(H);
    const long long np = H.n_p;
    const bool mg = H.inner_precond == SCHUR_INNER_MG;
    record_comp_means<double>(H, R, H.orr, 1);
    R.launch("cgS_init", k_cgS_init<T>, sgrid(H, np, k_cgS_init<T>), sblock(), H.g, C, v.invd,
             (const int*)H.cmpc, (const double*)H.cmean, H.orr, v.x, v.r, H.dctl, st,
             (const CgState*)&H.dctl->out, H.partials, (H.persistent || mg) ? -1 : s);
    if (mg) {
        record_mg_loop(H, R, true, sizeof(T) == sizeof(float), v.x, v.r, v.p, v.q, st,
                       (const int*)&H.dctl->out.skip_next);
    } else if (H.persistent) {
        R.launch_coop("cgS_loop", k_cgS_loop<T>, lgrid(H, np, k_cgS_loop<T>), sblock(), H.g, C,
                      v.invd, v.diag, v.x, v.r, v.p, v.q, H.dctl, st, H.partials,
                      (const int*)&H.dctl->out.skip_next);
    } else {
        R.loop(s, [&H, C, v, st, s, np](Recorder& B) {
            B.launch("cgS_dir", k_cgS_dir<T>, sgrid(H, np, k_cgS_dir<T>), sblock(), H.g, np, v.invd,
                     (const T*)v.r, v.p, H.dctl, (const CgState*)st);
            B.launch("cgS_matvec", k_cgS_matvec<T>, sgrid(H, np, k_cgS_matvec<T>), sblock(), H.g, C,
                     v.diag, (const T*)v.p, v.q, H.dctl, st, H.partials, s);
            B.launch("cgS_update", k_cgS_update<T>, sgrid(H, np, k_cgS_update<T>), sblock(), H.g, np,
                     v.invd, v.x, v.r, (const T*)v.p, (const T*)v.q, H.dctl, st, H.partials, s);
        });
    }
    record_comp_means<T>(H, R, (const T*)v.x, 0);
}

// Algorithm 1 in FP64.
static void record_solve_fp64(Handle& H, Recorder& R, int precond) {
    Ctl* ctl = H.dctl;
    CgState* inA = &ctl->inA;
    CgState* inS = &ctl->inS;
    const InnerA<double> A = innerA64(H);
    const InnerS<double> S = innerS64(H);
    const Compact C = compact_of(H);
    // slots are allocated before any loop body is recorded: in host-driven mode a body
    // runs once per iteration and must not allocate
    const int s_rhs = R.new_slot();
    const int s_out = R.new_slot();
    const int s_s0 = R.new_slot();
    const int s_a = R.new_slot();
    const int s_s = R.new_slot();
    record_A_solve<double>(H, R, A, inA, s_rhs, nullptr, 0.0, 1.0, nullptr);   // A^-1 f
    R.launch("outer_init", k_outer_init<double>, tgrid(H), tblock(), H.g, C, (const uint8_t*)H.mask,
             (const double*)A.x, H.og, H.orr, H.op, H.od, ctl, H.partials, s_out);
    if (precond == 1) {
        record_S_solve<double>(H, R, S, inS, s_s0);
        R.launch("outer_start", k_outer_start<double>, sgrid(H, H.n_p, k_outer_start<double>), sblock(), H.g, C,
                 (const int*)H.cmpc, (const double*)H.cmean, (const double*)S.x,
                 (const double*)H.orr, H.od, ctl, H.partials, s_out);
    }
    R.loop(s_out, [&H, C, ctl, inA, inS, A, S, precond, s_out, s_a, s_s](Recorder& B) {
        // q = S d = B A^-1 B^T d
        record_A_solve<double>(H, B, A, inA, s_a, H.od, 1.0, 0.0, nullptr);
        B.launch("outer_div", k_outer_div<double>, tgrid(H), tblock(), H.g, C, (const uint8_t*)H.mask,
                 (const double*)A.x, (const double*)H.od, H.oq, ctl, H.partials, s_out);
        B.launch("outer_update", k_outer_update, sgrid(H, H.g.ncell, k_outer_update), sblock(), H.g, H.op, H.orr,
                 (const double*)H.od, (const double*)H.oq, ctl, H.partials, s_out);
        if (precond == 1) {
            record_S_solve<double>(H, B, S, inS, s_s);
            B.launch("outer_dots", k_outer_dots<double>, sgrid(H, H.n_p, k_outer_dots<double>), sblock(), H.g, C,
                     (const int*)H.cmpc, (const double*)H.cmean, (const double*)S.x,
                     (const double*)H.orr, ctl, H.partials, s_out);
        }
        B.launch("outer_dir", k_outer_dir<double>, sgrid(H, H.g.ncell, k_outer_dir<double>), sblock(), H.g, C,
                 (const int*)H.cmpc, (const double*)H.cmean, (const double*)S.x,
                 (const double*)H.orr, H.od, ctl, (const int*)&ctl->out.done);
    });
}

// Mixed precision: FP64 defect correction around FP64 flexible CG with FP32 inner solves.
static void record_solve_mixed(Handle& H, Recorder& R, int precond) {
    Ctl* ctl = H.dctl;
    const InnerA<double> A64 = innerA64(H);
    const InnerA<float> A32 = innerA32(H);
    const InnerS<float> S32 = innerS32(H);
    const Compact C = compact_of(H);
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
    R.launch("outer_init", k_outer_init<double>, tgrid(H), tblock(), H.g, C, (const uint8_t*)H.mask,
             (const double*)A64.x, H.og, H.orr, H.op, H.od, ctl, H.partials, s_ref);
    R.loop(s_ref, [&H, C, ctl, A64, A32, S32, inA, inA32, inS32, precond, s_ref, s_s0, s_fcg, s_a,
                   s_s, s_t](Recorder& B) {
        if (precond == 1) record_S_solve<float>(H, B, S32, inS32, s_s0);
        B.launch("fcg_start", k_fcg_start<float>, sgrid(H, H.n_p, k_fcg_start<float>), sblock(), H.g, C,
                 (const int*)H.cmpc, (const double*)H.cmean, (const float*)S32.x,
                 (const double*)H.orr, H.od, ctl, H.partials, s_fcg);
        B.loop(s_fcg, [&H, C, ctl, A32, S32, inA32, inS32, precond, s_fcg, s_a, s_s,
                       s_ref](Recorder& D) {
            record_A_solve<float>(H, D, A32, inA32, s_a, H.od, 1.0, 0.0, nullptr);
            D.launch("fcg_div", k_fcg_div<float>, tgrid(H), tblock(), H.g, C, (const uint8_t*)H.mask,
                     (const float*)A32.x, (const double*)H.od, (const double*)H.orr, H.oq, ctl,
                     H.partials, s_fcg, s_ref);
            D.launch("fcg_update", k_fcg_update, sgrid(H, H.g.ncell, k_fcg_update), sblock(), H.g, H.op, H.orr,
                     (const double*)H.od, (const double*)H.oq, ctl, H.partials, s_fcg);
            if (precond == 1) record_S_solve<float>(H, D, S32, inS32, s_s);
            D.launch("fcg_dots", k_fcg_dots<float>, sgrid(H, H.n_p, k_fcg_dots<float>), sblock(), H.g, C,
                     (const int*)H.cmpc, (const double*)H.cmean, (const float*)S32.x,
                     (const double*)H.orr, (const double*)H.oq, ctl, H.partials);
            D.launch("fcg_dir", k_outer_dir<float>, sgrid(H, H.g.ncell, k_outer_dir<float>), sblock(), H.g, C,
                     (const int*)H.cmpc, (const double*)H.cmean, (const float*)S32.x,
                     (const double*)H.orr, H.od, ctl, (const int*)&ctl->out.skip_next);
        });
        // true residual with an FP64 inner solve: r = g - B A^-1 B^T p
        record_A_solve<double>(H, B, A64, inA, s_t, H.op, 1.0, 0.0, nullptr);
        B.launch("true_res", k_true_res, tgrid(H), tblock(), H.g, C, (const uint8_t*)H.mask,
                 (const double*)A64.x, (const double*)H.og, H.orr, ctl, H.partials, s_ref);
    });
}

void record_solve(Handle& H, Recorder& R, int precond, int precision) {
    if (precision == 1) record_solve_mixed(H, R, precond);
    else record_solve_fp64(H, R, precond);
}

void record_recover(Handle& H, Recorder& R) {
    Ctl* ctl = H.dctl;
    const int s = R.new_slot();
    record_A_solve<double>(H, R, innerA64(H), &ctl->rec, s, H.op, -1.0, 1.0, nullptr);
    R.launch("copy_u", k_copy_u, sgrid(H, H.n_u, k_copy_u), sblock(), H.g, compact_of(H),
             (const double*)H.ax, H.u, ctl, H.partials);
}

void record_solve_recover(Handle& H, Recorder& R, int precond, int precision) {
    record_solve(H, R, precond, precision);
    record_recover(H, R);
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
// Deterministic right-hand side for timing the SIMPLE loop: hashed values in [-0.5, 0.5).
__global__ void k_fill_pattern(double* __restrict__ v, long long n) {
    STREAM_LOOP(i, n) v[i] = (double)(((uint32_t)i * 2654435761u) >> 12) / 1048576.0 - 0.5;
}

// One cooperative launch of a persistent inner-CG kernel running exactly
// SCHUR_TIMED_LOOP_ITERS iterations (tolerance 0) from a fixed right-hand side: the A loop
// from b = f, the SIMPLE loop from a hashed cell vector.  Only the loop launch is timed.
template <typename T>
static cudaError_t time_loop_t(Handle& H, bool simple, InnerA<T> a, InnerS<T> sv, float* ms,
                               bool mg = false) {
    Ctl* ctl = H.dctl;
    CgState* st = &ctl->solo;
    const Compact C = compact_of(H);
    H.hctl->solo.tol = 0.0;
    H.hctl->solo.max_iter = SCHUR_TIMED_LOOP_ITERS;
    H.hctl->solo.skip_next = 0;
    cudaError_t e = cudaMemcpyAsync(&ctl->solo, &H.hctl->solo, sizeof(CgState),
                                    cudaMemcpyHostToDevice, H.stream);
    if (e != cudaSuccess) return e;
    const dim3 b = sblock();
    if (!simple) {
        k_cgA_init<T><<<sgrid(H, H.n_u, k_cgA_init<T>), b, 0, H.stream>>>(
            H.g, C, a.x, a.r, nullptr, 0.0, 1.0, nullptr, ctl, st, H.partials, -1);
    } else {
        k_fill_pattern<<<sgrid(H, H.g.ncell, k_fill_pattern), b, 0, H.stream>>>(H.orr, H.g.ncell);
        k_cgS_init<T><<<sgrid(H, H.n_p, k_cgS_init<T>), b, 0, H.stream>>>(
            H.g, C, sv.invd, H.cmpc, H.cmean, H.orr, sv.x, sv.r, ctl, st, st, H.partials, -1);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaEventRecord(H.ev0, H.stream)) != cudaSuccess) return e;
    if (mg) {
        int slot = kSlots - 1;
        Recorder R(H.stream, ctl, &slot);
        if (!simple)
            record_mg_loop(H, R, false, sizeof(T) == sizeof(float), a.x, a.r, a.p, a.q, st, nullptr);
        else
            record_mg_loop(H, R, true, sizeof(T) == sizeof(float), sv.x, sv.r, sv.p, sv.q, st, nullptr);
        if (!R.ok()) return R.error();
    } else if (!simple) {
        void* args[] = {(void*)&H.g, (void*)&C, (void*)&a.x, (void*)&a.r, (void*)&a.p, (void*)&a.q,
                        (void*)&ctl, (void*)&st, (void*)&H.partials};
        e = cudaLaunchCooperativeKernel((const void*)k_cgA_loop<T>, lgrid(H, H.n_u, k_cgA_loop<T>), b,
                                        args, 0, H.stream);
    } else {
        const int* gate = nullptr;
        void* args[] = {(void*)&H.g, (void*)&C, (void*)&sv.invd, (void*)&sv.diag, (void*)&sv.x,
                        (void*)&sv.r, (void*)&sv.p, (void*)&sv.q, (void*)&ctl, (void*)&st,
                        (void*)&H.partials, (void*)&gate};
        e = cudaLaunchCooperativeKernel((const void*)k_cgS_loop<T>, lgrid(H, H.n_p, k_cgS_loop<T>), b,
                                        args, 0, H.stream);
    }
    if (e != cudaSuccess) return e;
    if ((e = cudaEventRecord(H.ev1, H.stream)) != cudaSuccess) return e;
    if ((e = cudaEventSynchronize(H.ev1)) != cudaSuccess) return e;
    return cudaEventElapsedTime(ms, H.ev0, H.ev1);
}

static cudaError_t time_loop(Handle& H, int which, float* ms) {
    switch (which) {
        case 12: return time_loop_t<double>(H, false, innerA64(H), innerS64(H), ms);
        case 13: return time_loop_t<double>(H, true, innerA64(H), innerS64(H), ms);
        case 14: return time_loop_t<float>(H, false, innerA32(H), innerS32(H), ms);
        case 15: return time_loop_t<float>(H, true, innerA32(H), innerS32(H), ms);
        case 16: return time_loop_t<double>(H, false, innerA64(H), innerS64(H), ms, true);
        case 17: return time_loop_t<double>(H, true, innerA64(H), innerS64(H), ms, true);
        case 18: return time_loop_t<float>(H, false, innerA32(H), innerS32(H), ms, true);
        case 19: return time_loop_t<float>(H, true, innerA32(H), innerS32(H), ms, true);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t time_kernel(Handle& H, int which, int slot, float* ms) {
    if (!H.ev0) {
        cudaError_t e = cudaEventCreate(&H.ev0);
        if (e == cudaSuccess) e = cudaEventCreate(&H.ev1);
        if (e != cudaSuccess) return e;
    }
    if (((which >= 6 && which < 12) || which == 14 || which == 15 || which >= 18) && !H.axf)
        return cudaErrorInvalidValue;
    Ctl* ctl = H.dctl;
    CgState* st = &ctl->solo;
    const long long nu = H.n_u, np = H.n_p;
    const Compact C = compact_of(H);
    if (which >= 12) return time_loop(H, which, ms);
    cudaError_t e = cudaEventRecord(H.ev0, H.stream);
    if (e != cudaSuccess) return e;
    const dim3 b = sblock();
#define GU(k) sgrid(H, nu, k)
#define GP(k) sgrid(H, np, k)
    cudaStream_t s = H.stream;
    switch (which) {
        case 0: k_cgA_dir<double><<<GU(k_cgA_dir<double>), b, 0, s>>>(H.g, nu, H.ufl, H.ar, H.ap, ctl, st); break;
        case 1: k_cgA_matvec<double><<<GU(k_cgA_matvec<double>), b, 0, s>>>(H.g, C, H.ap, H.aq, ctl, st, H.partials, slot); break;
        case 2: k_cgA_update<double><<<GU(k_cgA_update<double>), b, 0, s>>>(H.g, nu, H.ufl, H.ax, H.ar, H.ap, H.aq, ctl, st, H.partials, slot); break;
        case 3: k_cgS_dir<double><<<GP(k_cgS_dir<double>), b, 0, s>>>(H.g, np, H.invdSc, H.sr, H.sp, ctl, st); break;
        case 4: k_cgS_matvec<double><<<GP(k_cgS_matvec<double>), b, 0, s>>>(H.g, C, H.dSc, H.sp, H.sq, ctl, st, H.partials, slot); break;
        case 5: k_cgS_update<double><<<GP(k_cgS_update<double>), b, 0, s>>>(H.g, np, H.invdSc, H.sx, H.sr, H.sp, H.sq, ctl, st, H.partials, slot); break;
        case 6: k_cgA_dir<float><<<GU(k_cgA_dir<float>), b, 0, s>>>(H.g, nu, H.ufl, H.arf, H.apf, ctl, st); break;
        case 7: k_cgA_matvec<float><<<GU(k_cgA_matvec<float>), b, 0, s>>>(H.g, C, H.apf, H.aqf, ctl, st, H.partials, slot); break;
        case 8: k_cgA_update<float><<<GU(k_cgA_update<float>), b, 0, s>>>(H.g, nu, H.ufl, H.axf, H.arf, H.apf, H.aqf, ctl, st, H.partials, slot); break;
        case 9: k_cgS_dir<float><<<GP(k_cgS_dir<float>), b, 0, s>>>(H.g, np, H.invdSf, H.srf, H.spf, ctl, st); break;
        case 10: k_cgS_matvec<float><<<GP(k_cgS_matvec<float>), b, 0, s>>>(H.g, C, (const float*)nullptr, H.spf, H.sqf, ctl, st, H.partials, slot); break;
        case 11: k_cgS_update<float><<<GP(k_cgS_update<float>), b, 0, s>>>(H.g, np, H.invdSf, H.sxf, H.srf, H.spf, H.sqf, ctl, st, H.partials, slot); break;
        default: return cudaErrorInvalidValue;
    }
#undef GU
#undef GP
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(H.ev1, H.stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(H.ev1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, H.ev0, H.ev1);
    return e;
}

// FP64 pipe throughput: 8 independent chains of dependent DFMAs per thread (the chains
// keep the pipe busy; the result is stored so that nothing is optimised away).
__global__ void k_dfma_peak(double* __restrict__ out, int iters, double x, double y) {
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fma(a[k], x, y);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

cudaError_t measure_fp64_peak(cudaStream_t s, int iters, double* lane_ops_per_s) {
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int blocks = nsm * 8, threads = 256;
    double* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMalloc((void**)&out, (size_t)blocks * threads * sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.0f;
    if (e == cudaSuccess) {
        // x slightly below 1 and y small keep every chain bounded and normal
        k_dfma_peak<<<blocks, threads, 0, s>>>(out, iters, 0.999999, 1e-6);   // warm-up
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        k_dfma_peak<<<blocks, threads, 0, s>>>(out, iters, 0.999999, 1e-6);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    if (e == cudaSuccess)
        *lane_ops_per_s = (double)blocks * threads * 8.0 * (double)iters / ((double)ms * 1e-3);
    return e;
}

cudaError_t launch_build_tables(Handle& H) {
    const Compact C = compact_of(H);
    if (H.n_u > 0)
        k_build_nbA<<<sgrid(H, H.n_u, k_build_nbA), sblock(), 0, H.stream>>>(H.g, C, H.nbA);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || H.n_p == 0) return e;
    k_build_nbS<<<sgrid(H, H.n_p, k_build_nbS), sblock(), 0, H.stream>>>(H.g, C, H.flags, H.nbS, H.codeS, H.dSc);
    return cudaGetLastError();
}

}  // namespace schur
