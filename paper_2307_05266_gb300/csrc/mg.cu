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
//   aggregates) counts as zero: the entry is a nullspace unknown with weight 0.
// V-cycle (from x = 0, on the residual r of the CG): z_l = omega D^-1 b_l and the residual
//   res_l = b_l - A_l z_l (one stencil on b), b_(l+1) = P^T res_l (a gather over the 8
//   children), the coarse correction scaled by gamma, and one Jacobi sweep after:
//   out_l = y + omega D^-1 (b_l - A_l y), y = z_l + gamma P out_(l+1) (one stencil whose
//   neighbour values are z at the neighbour plus the correction of its parent).  omega =
//   0.9; gamma = 1.3 (A) and 1.7 (S-hat).  The cycle is symmetric positive definite, the
//   CG stop rule is ||M^-1 r_k|| / ||M^-1 r_0|| < eps as for Jacobi, and the S-hat cycle's
//   output is not projected (r stays in the range; the solution is projected afterwards).
// Launch: one persistent cooperative kernel per inner solve.  The fine and the larger
//   coarse levels run on the whole grid with a grid barrier between phases; the levels
//   from `tail` down (at most kMgTailMax entries) run in block 0 alone with block barriers,
//   while the other blocks wait at one grid barrier.  Per CG iteration: matvec + p.q, the
//   x/r update, the V-cycle, z and the dots r.z, z.z, the direction update: 3 tail + 3 grid
//   barriers.  Every grid wait is bounded (grid_barrier).
#include <cstring>

#include "cg_dev.cuh"

namespace schur {

constexpr double kMgOmega = 0.9;
constexpr double kMgGammaA = 1.3;
constexpr double kMgGammaS = 1.7;
constexpr double kMgZeroDiag = 1e-12;
constexpr long long kMgTailMax = 1024;   // levels with at most this many entries: block 0
constexpr int kMgMaxLevels = 40;

// Device descriptor of one level.  Every vector has one more entry, kept at 0, that the
// sentinels of the tables point at (a missing neighbour, a missing child).  Level 0: b is
// the CG residual r, out is the CG's z (in its q buffer), and the operator comes from the
// fine tables (nb, ch, w, dg unused).  res holds the residual after pre-smoothing on the way
// down and, once the level above has used it, y = z + gamma P out_(l+1) on the way up.
template <typename T>
struct MgLev {
    uint32_t n, ld, nfine, ncoarse;
    const uint32_t* nb;   // [6][ld] neighbour entry per direction, n = none
    const uint32_t* ch;   // [8][ld] children at level l - 1, nfine = none
    const uint32_t* agg;  // [n + 1] parent at level l + 1 (agg[n] = ncoarse)
    const T* w;           // [6][ld] off-diagonal coefficients (0 at missing neighbours)
    const T* dg;          // [n] diagonal
    const T* wd;          // [n + 1] omega / diagonal (0: nullspace); last level: 1 / diagonal
    T* b;                 // [n + 1] right-hand side of the level
    T* z;                 // [n + 1] pre-smoothed correction wd b
    T* res;               // [n + 1] residual after pre-smoothing, then y
    T* out;               // level 0: the cycle's output
};

template <typename T>
struct MgRun {
    const MgLev<T>* lev;  // [nlev] device descriptors
    int nlev, tail;
    T gamma;
};

// ---- per-entry work of one phase ----------------------------------------------------------

// Fine operator of the compact layout applied at entry i to a vector v with v_i = vi.
template <typename T, bool kS>
__device__ __forceinline__ T fine_apply(const Tabs<T>& t, const Dev& g, const Compact& C,
                                        const T* __restrict__ dS, uint32_t i, T vi,
                                        const T* __restrict__ v) {
    const int ne = 2 * g.d;
    if constexpr (!kS) {
        const int gh = C.ufl[i] >> 1;
        T s = (T)0;
#pragma unroll
        for (int e = 0; e < 6; ++e)
            if (e < ne) s += v[__ldg(C.nbA + e * C.ldA + i)];
        return t.diag[gh] * vi - s;
    } else {
        const uint32_t code = __ldg(C.codeS + i);
        T s = (T)0;
        if constexpr (sizeof(T) == 8) {
#pragma unroll
            for (int e = 0; e < 6; ++e)
                if (e < ne) s += t.w[(code >> (3 * e)) & 7u] * v[__ldg(C.nbS + e * C.ldS + i)];
            return dS[i] * vi - s;
        } else {
#pragma unroll
            for (int e = 0; e < 6; ++e)
                if (e < ne) s += t.w[(code >> (3 * e)) & 7u] * (vi - v[__ldg(C.nbS + e * C.ldS + i)]);
            return s;
        }
    }
}

// Coarse operator of level L applied at entry i to v.
template <typename T>
__device__ __forceinline__ T coarse_apply(const MgLev<T>& L, uint32_t i, T vi, const T* __restrict__ v) {
    T s = L.dg[i] * vi;
#pragma unroll
    for (int e = 0; e < 6; ++e) s += L.w[e * L.ld + i] * v[__ldg(L.nb + e * L.ld + i)];
    return s;
}

// Prolongation of the correction of entry i of level L to its children: y = z + gamma out
// on the level below (written into that level's res buffer, whose residual is consumed).
template <typename T>
__device__ __forceinline__ void prolong_entry(const MgLev<T>& L, const T* __restrict__ zf,
                                              T* __restrict__ yf, T gamma, T out, uint32_t i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const uint32_t k = __ldg(L.ch + c * L.ld + i);
        if (k < L.nfine) yf[k] = zf[k] + gamma * out;
    }
}

// Fine level, down: res0 = r - Op z0 (z0 = wd0 r, formed with r).
template <typename T, bool kS>
__device__ __forceinline__ void mg_down_fine_entry(const Tabs<T>& t, const Dev& g, const Compact& C,
                                                   const T* __restrict__ dS, const MgLev<T>& L,
                                                   uint32_t i) {
    const T* __restrict__ z = L.z;
    L.res[i] = L.b[i] - fine_apply<T, kS>(t, g, C, dS, i, z[i], z);
}

// Fine level, up: z = y + wd0 (r - Op y); returns z (the CG's preconditioned residual,
// stored in out = q).
template <typename T, bool kS>
__device__ __forceinline__ T mg_up_fine_entry(const Tabs<T>& t, const Dev& g, const Compact& C,
                                              const T* __restrict__ dS, const MgLev<T>& L,
                                              uint32_t i) {
    const T* __restrict__ y = L.res;
    const T yi = y[i];
    const T zf = yi + L.wd[i] * (L.b[i] - fine_apply<T, kS>(t, g, C, dS, i, yi, y));
    L.out[i] = zf;
    return zf;
}

// Coarse level, down: res = b - A z.
template <typename T>
__device__ __forceinline__ void mg_down_entry(const MgLev<T>& L, uint32_t i) {
    const T* __restrict__ z = L.z;
    L.res[i] = L.b[i] - coarse_apply(L, i, z[i], z);
}

// Coarse level, restriction: b = the sum of the children's residuals, z = wd b; on the last
// level z is the exact solve and is prolonged at once.
template <typename T>
__device__ __forceinline__ void mg_restrict_entry(const MgLev<T>& L, const MgLev<T>& F, T gamma,
                                                  bool last, uint32_t i) {
    const T* __restrict__ resf = F.res;
    T s = (T)0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += resf[__ldg(L.ch + c * L.ld + i)];
    L.b[i] = s;
    const T zi = L.wd[i] * s;
    L.z[i] = zi;
    if (last) prolong_entry(L, (const T*)F.z, F.res, gamma, zi, i);
}

// Coarse level, up: out = y + wd (b - A y), prolonged to the level below.
template <typename T>
__device__ __forceinline__ void mg_up_entry(const MgLev<T>& L, const MgLev<T>& F, T gamma, uint32_t i) {
    const T* __restrict__ y = L.res;
    const T yi = y[i];
    const T out = yi + L.wd[i] * (L.b[i] - coarse_apply(L, i, yi, y));
    prolong_entry(L, (const T*)F.z, F.res, gamma, out, i);
}

// ---- loops over a level: the whole grid (grid-stride) or block 0 alone -----------------

#define MG_GRID_LOOP(i, n)                                                                  \
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += gridDim.x * blockDim.x)
#define MG_BLOCK_LOOP(i, n) for (uint32_t i = threadIdx.x; i < (n); i += blockDim.x)

// The multigrid-preconditioned CG loop of one inner solve, after its init kernel (x = 0,
// r = b, status NOTCONV when b != 0).  dS: the diagonal of S-hat (FP64 S stencil).  Same
// contract as the Jacobi loop kernels: all blocks hold bitwise-equal scalars (block-
// identical grid sums), `gate` skips the solve, block 0 writes the final state, a failed
// barrier leaves ST_BARRIER.
template <typename T, bool kS>
__device__ __forceinline__ void mg_loop(const Dev& g, const Compact& C, const MgRun<T>& M,
                                        const T* __restrict__ dS, T* __restrict__ xv,
                                        T* __restrict__ rv, T* __restrict__ pv, T* __restrict__ qv,
                                        Ctl* ctl, CgState* st, double* partials, const int* gate) {
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
    const int nlev = M.nlev, tail = M.tail;
    const T gamma = M.gamma;
    const T* __restrict__ wd0 = M.lev[0].wd;
    T* __restrict__ z0 = M.lev[0].z;
    unsigned target = 0;
    bool ok = true;
    bool started = false;
    // z0 = wd0 r for the first cycle (later cycles form it with the r update)
    MG_GRID_LOOP(i, n) z0[i] = wd0[i] * rv[i];
    for (;;) {
        // ---- V-cycle on r (r and z0 complete after this barrier)
        if (!(ok = grid_barrier(ctl, target))) break;
        {
            const MgLev<T> L0 = M.lev[0];
            MG_GRID_LOOP(i, n) mg_down_fine_entry<T, kS>(t, g, C, dS, L0, i);
        }
        if (!(ok = grid_barrier(ctl, target))) break;
        for (int l = 1; l < tail; ++l) {
            {
                const MgLev<T> L = M.lev[l], F = M.lev[l - 1];
                MG_GRID_LOOP(i, L.n) mg_restrict_entry<T>(L, F, gamma, false, i);
            }
            if (!(ok = grid_barrier(ctl, target))) break;
            {
                const MgLev<T> L = M.lev[l];
                MG_GRID_LOOP(i, L.n) mg_down_entry<T>(L, i);
            }
            if (!(ok = grid_barrier(ctl, target))) break;
        }
        if (!ok) break;
        if (blockIdx.x == 0) {
            for (int l = tail; l < nlev; ++l) {
                const MgLev<T> L = M.lev[l], F = M.lev[l - 1];
                const bool last = (l == nlev - 1);
                MG_BLOCK_LOOP(i, L.n) mg_restrict_entry<T>(L, F, gamma, last, i);
                __syncthreads();
                if (!last) {
                    MG_BLOCK_LOOP(i, L.n) mg_down_entry<T>(L, i);
                    __syncthreads();
                }
            }
            for (int l = nlev - 2; l >= tail; --l) {
                const MgLev<T> L = M.lev[l], F = M.lev[l - 1];
                MG_BLOCK_LOOP(i, L.n) mg_up_entry<T>(L, F, gamma, i);
                __syncthreads();
            }
        }
        if (!(ok = grid_barrier(ctl, target))) break;
        for (int l = tail - 1; l >= 1; --l) {
            {
                const MgLev<T> L = M.lev[l], F = M.lev[l - 1];
                MG_GRID_LOOP(i, L.n) mg_up_entry<T>(L, F, gamma, i);
            }
            if (!(ok = grid_barrier(ctl, target))) break;
        }
        if (!ok) break;
        // ---- z = the cycle's output (in q), r.z and z.z
        double v2[2];
        {
            const MgLev<T> L0 = M.lev[0];
            T a0 = (T)0, a1 = (T)0;
            MG_GRID_LOOP(i, n) {
                const T zf = mg_up_fine_entry<T, kS>(t, g, C, dS, L0, i);
                a0 += rv[i] * zf;
                a1 += zf * zf;
            }
            v2[0] = (double)a0;
            v2[1] = (double)a1;
        }
        if (!(ok = grid_sum<2>(v2, P2, ctl, target))) break;
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
        {
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
        // ---- x += alpha p, r -= alpha q, z0 = wd0 r (the first smoothing step)
        {
            const T alpha = (T)s.alpha;
            T* __restrict__ x = opaque(xv);
            T* __restrict__ r = opaque(rv);
            const T* __restrict__ p = opaque(pv);
            const T* __restrict__ q = opaque(qv);
            const T* __restrict__ w0 = opaque(wd0);
            T* __restrict__ zz = opaque(z0);
            MG_GRID_LOOP(i, n) {
                x[i] += alpha * p[i];
                const T ri = r[i] - alpha * q[i];
                r[i] = ri;
                zz[i] = w0[i] * ri;
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (!ok) s.status = ST_BARRIER;
        *st = s;
        note_inner_status(ctl, s.status);
    }
}

template <typename T, bool kS>
__global__ void __launch_bounds__(kBlock, 3) k_mg_loop(Dev g, Compact C, MgRun<T> M,
                                                       const T* __restrict__ dS, T* __restrict__ xv,
                                                       T* __restrict__ rv, T* __restrict__ pv,
                                                       T* __restrict__ qv, Ctl* ctl, CgState* st,
                                                       double* partials, const int* gate) {
    count_launch(ctl);
    mg_loop<T, kS>(g, C, M, dS, xv, rv, pv, qv, ctl, st, partials, gate);
}

// ---- hierarchy build (host) ---------------------------------------------------------------

namespace {

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
    for (long long k = 0; k < n; ++k) {
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
    for (long long i = 0; i < F.n; ++i) idx[key(F.a[i], F.x[i] >> 1, F.y[i] >> 1, F.z[i] >> 1)] = 0;
    long long nc = 0;
    C = HostLevel();
    C.dims[0] = cx;
    C.dims[1] = cy;
    C.dims[2] = cz;
    for (int a = 0; a < ncomp; ++a)
        for (int Z = 0; Z < cz; ++Z)
            for (int Y = 0; Y < cy; ++Y)
                for (int X = 0; X < cx; ++X) {
                    int32_t& v = idx[key(a, X, Y, Z)];
                    if (v < 0) continue;
                    v = (int32_t)nc++;
                    C.a.push_back((int8_t)a);
                    C.x.push_back((int16_t)X);
                    C.y.push_back((int16_t)Y);
                    C.z.push_back((int16_t)Z);
                }
    C.n = nc;
    C.ld = round_up(nc + 1, 32);
    agg.assign((size_t)F.n + 1, (uint32_t)nc);
    ch.assign((size_t)(8 * C.ld), (uint32_t)F.n);
    for (long long i = 0; i < F.n; ++i) {
        const uint32_t I = (uint32_t)idx[key(F.a[i], F.x[i] >> 1, F.y[i] >> 1, F.z[i] >> 1)];
        agg[i] = I;
        const int slot = (F.x[i] & 1) | ((F.y[i] & 1) << 1) | ((F.z[i] & 1) << 2);
        ch[slot * C.ld + I] = (uint32_t)i;
    }
    // coarse neighbours: the aggregate one step away along each direction (wrapped on a
    // periodic axis); a step that wraps onto the aggregate itself is a diagonal coupling
    const int cd[3] = {cx, cy, cz};
    C.nb.assign((size_t)(6 * C.ld), (uint32_t)nc);
    for (long long I = 0; I < nc; ++I)
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
    // Galerkin coefficients, summed over the fine entries in their order
    C.w.assign((size_t)(6 * C.ld), 0.0);
    C.dg.assign((size_t)nc, 0.0);
    C.mass.assign((size_t)nc, 0.0);
    for (long long i = 0; i < F.n; ++i) {
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
                if (C.nb[e * C.ld + I] != J) return false;
                C.w[e * C.ld + I] += c;
            }
        }
    }
    return true;
}

bool single_cell(const HostLevel& L) {
    for (long long i = 0; i < L.n; ++i)
        if (L.x[i] || L.y[i] || L.z[i]) return false;
    return true;
}

// Weights of the smoother (omega / diagonal) or, on the last level, of the exact solve
// (1 / diagonal); 0 for a diagonal that counts as zero; one more entry (0) for the sentinel.
std::vector<double> weights(const HostLevel& L, double scale) {
    std::vector<double> wd((size_t)L.n + 1, 0.0);
    for (long long i = 0; i < L.n; ++i)
        if (L.dg[i] > kMgZeroDiag * L.mass[i]) wd[i] = scale / L.dg[i];
    return wd;
}

template <typename T>
__global__ void k_mg_convert(const double* __restrict__ src, T* __restrict__ dst, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = (T)src[i];
}

// Device descriptors of precision T over the hierarchy's tables (FP32 values converted from
// the FP64 ones; vectors allocated per precision).
template <typename T>
int build_descriptors(Handle& H, MgOp& M, bool simple, void** out) {
    const int L = M.nlev;
    const cudaStream_t s = H.stream;
    std::vector<MgLev<T>> d((size_t)L);
    cudaError_t e = cudaSuccess;
    auto conv = [&](const double* src, long long n, const T** dst) {
        if (e != cudaSuccess) return;
        if (sizeof(T) == sizeof(double)) {
            *dst = (const T*)src;
            return;
        }
        T* p = nullptr;
        e = mg_alloc(M, s, &p, (size_t)n);
        if (e != cudaSuccess) return;
        k_mg_convert<T><<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, s>>>(src, p, n);
        e = cudaGetLastError();
        *dst = p;
    };
    auto vec = [&](long long n, T** dst) {
        if (e == cudaSuccess) e = mg_alloc(M, s, dst, (size_t)n);
    };
    const bool f32 = sizeof(T) == sizeof(float);
    for (int l = 0; l < L; ++l) {
        MgLev<T>& v = d[l];
        std::memset(&v, 0, sizeof(v));
        v.n = (uint32_t)M.n[l];
        v.ld = (uint32_t)M.ld[l];
        v.nfine = l > 0 ? (uint32_t)M.n[l - 1] : 0u;
        v.ncoarse = l + 1 < L ? (uint32_t)M.n[l + 1] : 0u;
        v.nb = M.nb[l];
        v.ch = M.ch[l];
        v.agg = M.agg[l];
        if (l > 0) {
            conv(M.w[l], 6 * M.ld[l], &v.w);
            conv(M.dg[l], M.n[l], &v.dg);
        }
        conv(M.wd[l], M.n[l] + 1, &v.wd);
        if (l == 0) {
            // the CG's own vectors: b = r (one zero entry past the end), out = q
            v.b = simple ? (f32 ? (T*)H.srf : (T*)H.sr) : (f32 ? (T*)H.arf : (T*)H.ar);
            v.out = simple ? (f32 ? (T*)H.sqf : (T*)H.sq) : (f32 ? (T*)H.aqf : (T*)H.aq);
        } else {
            vec(M.n[l] + 1, &v.b);
        }
        vec(M.n[l] + 1, &v.z);
        vec(M.n[l] + 1, &v.res);
    }
    MgLev<T>* dev = nullptr;
    if (e == cudaSuccess) e = mg_alloc(M, s, &dev, (size_t)L);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dev, d.data(), (size_t)L * sizeof(MgLev<T>), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaErrorMemoryAllocation)
        return schur_set_error_internal(SCHUR_ENOMEM, "device allocation failed");
    if (e != cudaSuccess) return schur_set_error_internal(SCHUR_ECUDA, cudaGetErrorString(e));
    *out = dev;
    return SCHUR_OK;
}

int build_hierarchy(Handle& H, MgOp& M, bool simple) {
    const Dev& g = H.g;
    const cudaStream_t s = H.stream;
    cudaError_t e = cudaStreamSynchronize(s);   // the fine tables are complete
    const int ncomp = simple ? 1 : g.d;
    std::vector<HostLevel> lv(1);
    if (e == cudaSuccess) e = fine_level(H, simple, lv[0]);
    if (e != cudaSuccess) return schur_set_error_internal(SCHUR_ECUDA, cudaGetErrorString(e));
    std::vector<std::vector<uint32_t>> aggs, chs(1);
    do {   // at least one coarse level, until the grid is a single cell
        HostLevel c;
        std::vector<uint32_t> agg, ch;
        if (!coarsen(lv.back(), g.per, ncomp, c, agg, ch))
            return schur_set_error_internal(SCHUR_ECUDA, "multigrid: inconsistent coarse coupling");
        aggs.push_back(std::move(agg));
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
    M.ld.assign(L, 0);
    M.nb.assign(L, nullptr);
    M.ch.assign(L, nullptr);
    M.agg.assign(L, nullptr);
    M.w.assign(L, nullptr);
    M.dg.assign(L, nullptr);
    M.wd.assign(L, nullptr);
    M.tail = L - 1;
    for (int l = 1; l < L; ++l)
        if (lv[l].n <= kMgTailMax) {
            M.tail = l;
            break;
        }
    for (int l = 0; l < L && e == cudaSuccess; ++l) {
        const HostLevel& v = lv[l];
        M.n[l] = v.n;
        M.ld[l] = v.ld;
        if (l + 1 < L) e = upload(M, s, &M.agg[l], aggs[l]);
        const bool last = (l == L - 1);
        if (e == cudaSuccess) e = upload(M, s, &M.wd[l], weights(v, last ? 1.0 : kMgOmega));
        if (l == 0 || e != cudaSuccess) continue;
        e = upload(M, s, &M.nb[l], v.nb);
        if (e == cudaSuccess) e = upload(M, s, &M.ch[l], chs[l]);
        if (e == cudaSuccess) e = upload(M, s, &M.w[l], v.w);
        if (e == cudaSuccess) e = upload(M, s, &M.dg[l], v.dg);
    }
    if (e == cudaErrorMemoryAllocation)
        return schur_set_error_internal(SCHUR_ENOMEM, "device allocation failed");
    if (e != cudaSuccess) return schur_set_error_internal(SCHUR_ECUDA, cudaGetErrorString(e));
    return build_descriptors<double>(H, M, simple, &M.lev64);
}

}  // namespace

void mg_free(MgOp& M) {
    for (void* p : M.bufs) cudaFree(p);
    M = MgOp();
}

int mg_prepare(Handle& H, bool simple, bool fp32) {
    MgOp& M = simple ? H.mgS : H.mgA;
    if ((simple ? H.n_p : H.n_u) == 0) return SCHUR_OK;   // nothing to solve
    if (!M.nlev) {
        const long long before = M.bytes;
        const int rc = build_hierarchy(H, M, simple);
        if (rc) {
            mg_free(M);
            return rc;
        }
        H.bytes += M.bytes - before;
    }
    if (fp32 && !M.lev32) {
        const long long before = M.bytes;
        const int rc = build_descriptors<float>(H, M, simple, &M.lev32);
        if (rc) return rc;
        H.bytes += M.bytes - before;
    }
    return SCHUR_OK;
}

void record_mg_loop(Handle& H, Recorder& R, bool simple, bool fp32, void* x, void* r, void* p,
                    void* q, CgState* st, const int* gate) {
    const MgOp& M = simple ? H.mgS : H.mgA;
    const Compact C = compact_of(H);
    const long long n = simple ? H.n_p : H.n_u;
    if (!M.nlev) return;   // no entries: the init kernel already finished the solve
    if (!fp32) {
        MgRun<double> run{(const MgLev<double>*)M.lev64, M.nlev, M.tail,
                          simple ? kMgGammaS : kMgGammaA};
        if (simple)
            R.launch_coop("mgS_loop", k_mg_loop<double, true>, lgrid(H, n, k_mg_loop<double, true>),
                          sblock(), H.g, C, run, (const double*)H.dSc, (double*)x, (double*)r,
                          (double*)p, (double*)q, H.dctl, st, H.partials, gate);
        else
            R.launch_coop("mgA_loop", k_mg_loop<double, false>, lgrid(H, n, k_mg_loop<double, false>),
                          sblock(), H.g, C, run, (const double*)nullptr, (double*)x, (double*)r,
                          (double*)p, (double*)q, H.dctl, st, H.partials, gate);
    } else {
        MgRun<float> run{(const MgLev<float>*)M.lev32, M.nlev, M.tail,
                         (float)(simple ? kMgGammaS : kMgGammaA)};
        if (simple)
            R.launch_coop("mgS_loop_f32", k_mg_loop<float, true>, lgrid(H, n, k_mg_loop<float, true>),
                          sblock(), H.g, C, run, (const float*)nullptr, (float*)x, (float*)r,
                          (float*)p, (float*)q, H.dctl, st, H.partials, gate);
        else
            R.launch_coop("mgA_loop_f32", k_mg_loop<float, false>, lgrid(H, n, k_mg_loop<float, false>),
                          sblock(), H.g, C, run, (const float*)nullptr, (float*)x, (float*)r,
                          (float*)p, (float*)q, H.dctl, st, H.partials, gate);
    }
}

}  // namespace schur
