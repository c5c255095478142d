// C ABI of the solver: handle lifetime, device memory, graph instantiation and launch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/schur.h"
#include "internal.h"

using namespace schur;

struct schur_geom {
    Handle H;
};

namespace {

thread_local std::string g_last_error;

int set_error(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int cuda_error(cudaError_t e, const char* what) {
    return set_error(SCHUR_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CUDA_TRY(expr, what)                                  \
    do {                                                      \
        cudaError_t e_ = (expr);                              \
        if (e_ != cudaSuccess) return cuda_error(e_, what);   \
    } while (0)

constexpr int kHostSlotBase = 24;
constexpr long long kMaxCompact = (1ll << 31) - (1ll << 24);
constexpr int kHistMax = 1 << 17;  // outer iterations kept in the per-iteration record

// Eigenvalues of the symmetric tridiagonal matrix (diagonal d[0..m), off-diagonal
// e[0..m-1)) below x: the number of negative pivots of the LDL^T factorisation of T - x I
// (Sturm sequence count).
long long sturm_count(const std::vector<double>& d, const std::vector<double>& e, double x) {
    long long cnt = 0;
    double q = 1.0;
    for (size_t i = 0; i < d.size(); ++i) {
        const double off = i ? e[i - 1] * e[i - 1] : 0.0;
        q = d[i] - x - (i ? off / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

// The k-th smallest eigenvalue (k = 0 .. m-1) of the tridiagonal matrix by bisection on
// the Sturm count inside the Gershgorin interval.
double tridiag_eig(const std::vector<double>& d, const std::vector<double>& e, long long k) {
    const size_t m = d.size();
    double lo = d[0], hi = d[0];
    for (size_t i = 0; i < m; ++i) {
        const double r = (i ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(e[i]) : 0.0);
        lo = std::min(lo, d[i] - r);
        hi = std::max(hi, d[i] + r);
    }
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (sturm_count(d, e, mid) > k) hi = mid; else lo = mid;
    }
    return 0.5 * (lo + hi);
}  // host-driven loops reuse slots 24..31 on every call

template <class T>
cudaError_t alloc(Handle& H, T** p, size_t n) {
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T) + 16);
    if (e == cudaSuccess) {
        H.bytes += (long long)(n * sizeof(T));
        e = cudaMemsetAsync(*p, 0, n * sizeof(T), H.stream);
    }
    return e;
}

void drop_graphs(Handle& H) {
    for (int k = 0; k < 4; ++k) {
        if (H.exec_solve[k]) cudaGraphExecDestroy(H.exec_solve[k]);
        if (H.graph_solve[k]) cudaGraphDestroy(H.graph_solve[k]);
        if (H.exec_full[k]) cudaGraphExecDestroy(H.exec_full[k]);
        if (H.graph_full[k]) cudaGraphDestroy(H.graph_full[k]);
        H.exec_solve[k] = H.exec_full[k] = nullptr;
        H.graph_solve[k] = H.graph_full[k] = nullptr;
    }
    if (H.exec_recover) cudaGraphExecDestroy(H.exec_recover);
    if (H.graph_recover) cudaGraphDestroy(H.graph_recover);
    if (H.exec_solo) cudaGraphExecDestroy(H.exec_solo);
    if (H.graph_solo) cudaGraphDestroy(H.graph_solo);
    H.exec_recover = H.exec_solo = nullptr;
    H.graph_recover = H.graph_solo = nullptr;
}

void free_all(Handle& H) {
    drop_graphs(H);
    if (H.done_ev) cudaEventDestroy(H.done_ev);
    H.done_ev = nullptr;
    void* bufs[] = {H.mask, H.flags, H.invdS, H.ax, H.ar, H.ap, H.aq, H.sx, H.sr, H.sp,
                    H.sq, H.op, H.orr, H.od, H.oq, H.og, H.u, H.partials, H.dctl,
                    H.cmpc, H.cmean, H.small_start, H.small_cells, H.ulist, H.flist,
                    H.axf, H.arf, H.apf, H.aqf, H.sxf, H.srf, H.spf, H.sqf, H.invdSf,
                    H.ufl, H.fmask, H.fbase, H.cmask, H.cbase, H.invdSc, H.stage,
                    H.nbA, H.nbS, H.codeS, H.dSc, H.hist};
    for (void* b : bufs)
        if (b) cudaFree(b);
    mg_free(H.mgA);
    mg_free(H.mgS);
    if (H.hctl) cudaFreeHost(H.hctl);
    if (H.ev0) cudaEventDestroy(H.ev0);
    if (H.ev1) cudaEventDestroy(H.ev1);
}

// Connected fluid components (two fluid cells are connected when the face between them
// is an unknown; periodic axes wrap), labelled on the host by union-find with the
// smaller index as root, so labels do not depend on the visiting order.  The largest
// components (at most kMaxBig, each of at least kBigMin cells) get ids 0..n_big-1 and are
// reduced by the whole grid; every other component is summed by one warp over its cell
// list.  Uploads cmp, small_start, small_cells and allocates cmean.
int build_components(Handle& H, const uint8_t* m) {
    const Dev& g = H.g;
    const long long n = g.ncell;
    std::vector<int> parent((size_t)n);
    for (long long c = 0; c < n; ++c) parent[c] = (m[c] == 1) ? (int)c : -1;
    auto find = [&](int x) {
        while (parent[x] != x) {
            parent[x] = parent[parent[x]];
            x = parent[x];
        }
        return x;
    };
    auto unite = [&](int a, int b) {
        a = find(a);
        b = find(b);
        if (a == b) return;
        if (a < b) parent[b] = a; else parent[a] = b;
    };
    for (int z = 0; z < g.nz; ++z)
        for (int y = 0; y < g.ny; ++y)
            for (int x = 0; x < g.nx; ++x) {
                const long long c = ((long long)z * g.ny + y) * g.nx + x;
                if (m[c] != 1) continue;
                for (int a = 0; a < g.d; ++a) {
                    int lx = x - (a == 0), ly = y - (a == 1), lz = z - (a == 2);
                    if (lx < 0) { if (!g.per[0]) continue; lx += g.nx; }
                    if (ly < 0) { if (!g.per[1]) continue; ly += g.ny; }
                    if (lz < 0) { if (!g.per[2]) continue; lz += g.nz; }
                    const long long l = ((long long)lz * g.ny + ly) * g.nx + lx;
                    if (m[l] == 1) unite((int)c, (int)l);
                }
            }
    std::vector<int> first_id((size_t)n, -1);
    std::vector<long long> size;
    std::vector<int> comp((size_t)n, -1);
    for (long long c = 0; c < n; ++c) {
        if (parent[c] < 0) continue;
        const int r = find((int)c);
        if (r == c) {
            first_id[c] = (int)size.size();
            size.push_back(0);
        }
        comp[c] = first_id[r];
        size[comp[c]]++;
    }
    const int ncomp = (int)size.size();
    std::vector<int> order(ncomp);
    std::iota(order.begin(), order.end(), 0);
    const int ntop = std::min(ncomp, kMaxBig);
    std::partial_sort(order.begin(), order.begin() + ntop, order.end(), [&](int a, int b) {
        return size[a] != size[b] ? size[a] > size[b] : a < b;
    });
    std::vector<int> remap(ncomp, -1);
    int nbig = 0;
    for (int i = 0; i < ntop; ++i)
        if (size[order[i]] >= kBigMin) {
            H.hctl->big_size[nbig] = (double)size[order[i]];
            remap[order[i]] = nbig++;
        }
    int next = nbig;
    for (int k = 0; k < ncomp; ++k)
        if (remap[k] < 0) remap[k] = next++;
    const int nsmall = ncomp - nbig;
    // compact cell order: fluid cells in C order (the order of flist)
    std::vector<uint32_t> fl;
    std::vector<int> cmpc;
    for (long long c = 0; c < n; ++c)
        if (comp[c] >= 0) {
            comp[c] = remap[comp[c]];
            fl.push_back((uint32_t)c);
            cmpc.push_back(comp[c]);
        }
    std::vector<int> start((size_t)nsmall + 1, 0);
    for (int k : cmpc)
        if (k >= nbig) start[k - nbig + 1]++;
    for (int j = 0; j < nsmall; ++j) start[j + 1] += start[j];
    std::vector<int> cells((size_t)std::max(start[nsmall], 1));
    std::vector<int> fill(start.begin(), start.end() - 1);
    for (size_t mi = 0; mi < cmpc.size(); ++mi)
        if (cmpc[mi] >= nbig) cells[fill[cmpc[mi] - nbig]++] = (int)mi;
    // compact face order (a, z, y, x) and the row bitmaps of faces and cells
    const int W = (g.nx + 31) / 32;
    const long long frows = (long long)g.d * g.nz * g.ny, crows = (long long)g.nz * g.ny;
    std::vector<uint32_t> ul, fmask((size_t)(frows * W), 0u), fbase((size_t)(frows * W), 0u);
    std::vector<uint32_t> cmask((size_t)(crows * W), 0u), cbase((size_t)(crows * W), 0u);
    for (int a = 0; a < g.d; ++a)
        for (int z = 0; z < g.nz; ++z)
            for (int y = 0; y < g.ny; ++y) {
                const long long row = ((long long)a * g.nz + z) * g.ny + y;
                for (int x = 0; x < g.nx; ++x) {
                    if ((x & 31) == 0) fbase[row * W + (x >> 5)] = (uint32_t)ul.size();
                    const long long c = ((long long)z * g.ny + y) * g.nx + x;
                    if (m[c] != 1) continue;
                    int lx = x - (a == 0), ly = y - (a == 1), lz = z - (a == 2);
                    if (lx < 0) { if (!g.per[0]) continue; lx += g.nx; }
                    if (ly < 0) { if (!g.per[1]) continue; ly += g.ny; }
                    if (lz < 0) { if (!g.per[2]) continue; lz += g.nz; }
                    const long long l = ((long long)lz * g.ny + ly) * g.nx + lx;
                    if (m[l] != 1) continue;
                    fmask[row * W + (x >> 5)] |= 1u << (x & 31);
                    ul.push_back((uint32_t)(a * g.stride + c));
                }
            }
    {
        uint32_t cnt = 0;
        for (long long row = 0; row < crows; ++row)
            for (int x = 0; x < g.nx; ++x) {
                if ((x & 31) == 0) cbase[row * W + (x >> 5)] = cnt;
                if (m[row * g.nx + x] == 1) {
                    cmask[row * W + (x >> 5)] |= 1u << (x & 31);
                    ++cnt;
                }
            }
    }
    H.n_u = (long long)ul.size();
    H.n_p = (long long)fl.size();
    // the inner kernels index compact vectors with 32-bit offsets (plus a grid's stride)
    if (H.n_u > kMaxCompact || H.n_p > kMaxCompact)
        return set_error(SCHUR_EINVAL, "more than 2^31 - 2^24 unknown faces or fluid cells");
    H.W = W;
    if (ul.empty()) ul.push_back(0);
    if (fl.empty()) { fl.push_back(0); cmpc.push_back(0); }
    H.n_comp = ncomp;
    H.n_big = nbig;
    H.n_small = nsmall;
    const size_t nu = ul.size(), np = fl.size();
    cudaError_t e = cudaSuccess;
    auto up = [&](auto** dst, const auto& src) {
        if (e == cudaSuccess) e = alloc(H, dst, src.size());
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(src[0]), cudaMemcpyHostToDevice,
                                H.stream);
    };
    up(&H.cmpc, cmpc);
    up(&H.small_start, start);
    up(&H.small_cells, cells);
    up(&H.ulist, ul);
    up(&H.flist, fl);
    up(&H.fmask, fmask);
    up(&H.fbase, fbase);
    up(&H.cmask, cmask);
    up(&H.cbase, cbase);
    auto A = [&](auto** p, size_t cnt) { if (e == cudaSuccess) e = alloc(H, p, cnt); };
    A(&H.cmean, (size_t)std::max(ncomp, 1));
    A(&H.ufl, nu);
    A(&H.invdSc, np);
    A(&H.dSc, np);
    // p vectors carry one more entry, kept at 0, that missing stencil neighbours point at
    // (r also: the multigrid smoother gathers r at stencil neighbours)
    A(&H.ax, nu); A(&H.ar, nu + 1); A(&H.ap, nu + 1); A(&H.aq, nu);
    A(&H.sx, np); A(&H.sr, np + 1); A(&H.sp, np + 1); A(&H.sq, np);
    H.ldA = (long long)(nu + 31) / 32 * 32;
    H.ldS = (long long)(np + 31) / 32 * 32;
    A(&H.nbA, (size_t)(2 * g.d * H.ldA));
    A(&H.nbS, (size_t)(2 * g.d * H.ldS));
    A(&H.codeS, np);
    if (e == cudaSuccess) e = launch_gather_u8(H, H.flags, H.ulist, H.ufl, (long long)nu);
    if (e == cudaSuccess) e = launch_gather_f64(H, H.invdS, H.flist, H.invdSc, (long long)np);
    if (e == cudaSuccess) e = launch_build_tables(H);
    if (e == cudaSuccess) e = cudaStreamSynchronize(H.stream);  // host vectors go out of scope
    if (e == cudaErrorMemoryAllocation) return set_error(SCHUR_ENOMEM, "device allocation failed");
    if (e != cudaSuccess) return cuda_error(e, "component upload");
    return SCHUR_OK;
}

// Build and instantiate one graph with recorder function `rec`.
template <class F>
int build_graph(Handle& H, cudaGraph_t* graph, cudaGraphExec_t* exec, F rec) {
    if (*exec) return SCHUR_OK;
    CUDA_TRY(cudaGraphCreate(graph, 0), "cudaGraphCreate");
    const size_t before = H.handles.size();
    Recorder R(*graph, H.dctl, &H.next_slot, &H.handles);
    rec(R);
    if (!R.ok()) return cuda_error(R.error(), ("graph recording: " + R.where()).c_str());
    for (size_t k = before; k < H.handles.size(); ++k)
        H.hctl->handle[H.handles[k].first] = H.handles[k].second;
    CUDA_TRY(cudaGraphInstantiate(exec, *graph, 0), "cudaGraphInstantiate");
    return SCHUR_OK;
}

void reset_call(Handle& H, int use_graph) {
    Ctl* c = H.hctl;
    c->use_graph = use_graph;
    c->f[0] = H.force[0];
    c->f[1] = H.force[1];
    c->f[2] = H.force[2];
    c->launches = 0;
    c->inner_status = 0;
    c->bar_count = 0;
    c->bar_err = 0;
    c->ticket = 0;
    c->inA.total = c->inS.total = c->out.total = c->solo.total = c->rec.total = 0;
    c->inA32.total = c->inS32.total = 0;
}

int upload(Handle& H) {
    CUDA_TRY(cudaMemcpyAsync(H.dctl, H.hctl, sizeof(Ctl), cudaMemcpyHostToDevice, H.stream),
             "control upload");
    return SCHUR_OK;
}

int download(Handle& H) {
    CUDA_TRY(cudaMemcpyAsync(H.hctl, H.dctl, sizeof(Ctl), cudaMemcpyDeviceToHost, H.stream),
             "control download");
    CUDA_TRY(cudaStreamSynchronize(H.stream), "stream synchronize");
    return SCHUR_OK;
}

// Status of a finished call: a failed grid barrier in any inner solve (ctl->bar_err)
// overrides the Krylov statuses, whose values are then meaningless.
int map_status(int st);

int call_status(const Ctl* c, int st) {
    if (c->bar_err) return SCHUR_ECUDA;
    return map_status(st);
}

const char* status_text(const Handle& H, const char* otherwise) {
    return H.hctl->bar_err ? "an inner-solve grid barrier wait ran past its limit (blocks of a "
                             "cooperative launch were not co-resident)"
                           : otherwise;
}

int map_status(int st) {
    if (st == ST_OK) return SCHUR_OK;
    if (st == ST_BREAKDOWN) return SCHUR_EBREAKDOWN;
    if (st == ST_BARRIER) return SCHUR_ECUDA;
    return SCHUR_ENOTCONV;
}

}  // namespace

int schur_set_error_internal(int code, const char* msg) { return set_error(code, msg); }

namespace schur {

Handle& handle_of(schur_geom_t g) { return g->H; }

int set_launch_shape(Handle& H, int blocks_per_sm, int entries_per_thread, int persistent) {
    if (blocks_per_sm < 1 || blocks_per_sm > 32 || entries_per_thread < 1 ||
        entries_per_thread > 4096 || (persistent != 0 && persistent != 1))
        return set_error(SCHUR_EINVAL, "blocks_per_sm must lie in [1, 32], entries_per_thread "
                                       "in [1, 4096] and persistent_inner in {0, 1}");
    if (H.pending) return set_error(SCHUR_ESTATE, "an asynchronous solve is in flight");
    const int tb = std::min(kMaxBlocks, H.nsm * blocks_per_sm);
    if (tb != H.target_blocks || entries_per_thread != H.min_per_thread ||
        (persistent != 0) != H.persistent) {
        cudaStreamSynchronize(H.stream);  // recorded graphs may still run
        drop_graphs(H);
        H.target_blocks = tb;
        H.min_per_thread = entries_per_thread;
        H.persistent = persistent != 0;
    }
    return SCHUR_OK;
}

schur_opts resolve_precond(const Handle& H, schur_opts o) {
    if (o.precond == SCHUR_PRECOND_AUTO)
        o.precond = (double)H.n_p < SCHUR_AUTO_SIMPLE_BELOW * (double)H.g.ncell ? SCHUR_SIMPLE
                                                                               : SCHUR_UZAWA;
    return o;
}

int check_opts(const schur_opts& o) {
    if (o.precond != SCHUR_UZAWA && o.precond != SCHUR_SIMPLE && o.precond != SCHUR_PRECOND_AUTO)
        return set_error(SCHUR_EINVAL, "precond must be SCHUR_UZAWA, SCHUR_SIMPLE or "
                                       "SCHUR_PRECOND_AUTO");
    if (o.stop_norm != SCHUR_STOP_UNPRECOND && o.stop_norm != SCHUR_STOP_PRECOND)
        return set_error(SCHUR_EINVAL, "bad stop_norm");
    if (o.precision != SCHUR_FP64 && o.precision != SCHUR_MIXED)
        return set_error(SCHUR_EINVAL, "precision must be SCHUR_FP64 or SCHUR_MIXED");
    if (o.precision == SCHUR_MIXED &&
        (!(o.tol_inner_f32 > 0) || !(o.refine_factor > 0 && o.refine_factor < 1) ||
         o.max_refine < 1 || o.step_max < 1))
        return set_error(SCHUR_EINVAL, "mixed precision needs tol_inner_f32 > 0, "
                                       "0 < refine_factor < 1, max_refine >= 1, step_max >= 1");
    if (o.loop_mode != SCHUR_LOOP_GRAPH && o.loop_mode != SCHUR_LOOP_HOST)
        return set_error(SCHUR_EINVAL, "bad loop_mode");
    if (o.inner_precond != SCHUR_INNER_JACOBI && o.inner_precond != SCHUR_INNER_MG)
        return set_error(SCHUR_EINVAL, "inner_precond must be SCHUR_INNER_JACOBI or SCHUR_INNER_MG");
    if (!(o.tol > 0) || !(o.tol_inner_A > 0) || !(o.tol_inner_S > 0) || o.max_outer < 1 ||
        o.max_inner < 1)
        return set_error(SCHUR_EINVAL, "tolerances must be > 0 and caps >= 1");
    return SCHUR_OK;
}

// Allocate what the options need and write them into the host control block (the
// recovery's inner solve uses the same tolerance and cap as the solve's A solves).
int prepare_solve(Handle& H, const schur_opts& opts, int use_graph) {
    const schur_opts o = resolve_precond(H, opts);  // the control block holds 0 or 1
    if (o.precision == SCHUR_MIXED && !H.axf) {
        // FP32 inner-solve buffers, allocated on the first mixed-precision solve
        const size_t nu = (size_t)std::max(H.n_u, 1ll), np = (size_t)std::max(H.n_p, 1ll);
        cudaError_t e = cudaSuccess;
        auto A = [&](float** p, size_t n) { if (e == cudaSuccess) e = alloc(H, p, n); };
        A(&H.axf, nu); A(&H.arf, nu + 1); A(&H.apf, nu + 1); A(&H.aqf, nu);
        A(&H.sxf, np); A(&H.srf, np + 1); A(&H.spf, np + 1); A(&H.sqf, np); A(&H.invdSf, np);
        if (e == cudaSuccess) e = launch_to_float(H, H.invdSc, H.invdSf, (long long)np);
        if (e == cudaErrorMemoryAllocation) return set_error(SCHUR_ENOMEM, "device allocation failed");
        if (e != cudaSuccess) return cuda_error(e, "mixed-precision buffers");
    }
    // inner preconditioner: the recorded graphs embed it, so a change drops them; the
    // multigrid hierarchies are built on first use (A always, S-hat for SIMPLE)
    if (o.inner_precond != H.inner_precond) {
        cudaStreamSynchronize(H.stream);  // recorded graphs may still run
        drop_graphs(H);
        H.inner_precond = o.inner_precond;
    }
    if (o.inner_precond == SCHUR_INNER_MG) {
        int rc = mg_prepare(H, false);
        if (!rc && o.precond == SCHUR_SIMPLE) rc = mg_prepare(H, true);
        if (rc) return rc;
    }
    // per-iteration record of the outer loop, NaN-filled (all bytes 0xff) before the call
    const int need = std::min(std::max(o.max_outer, 1), kHistMax);
    if (H.hist_cap < need) {
        if (H.hist) cudaFree(H.hist);
        H.hist = nullptr;
        H.hist_cap = 0;
        cudaError_t e = cudaMalloc((void**)&H.hist, (size_t)need * 4 * sizeof(double));
        if (e == cudaErrorMemoryAllocation) return set_error(SCHUR_ENOMEM, "device allocation failed");
        if (e != cudaSuccess) return cuda_error(e, "history buffer");
        H.hist_cap = need;
    }
    CUDA_TRY(cudaMemsetAsync(H.hist, 0xff, (size_t)need * 4 * sizeof(double), H.stream),
             "history reset");
    Ctl* c = H.hctl;
    reset_call(H, use_graph);
    c->hist = H.hist;
    c->hist_cap = need;
    c->precond = o.precond;
    c->stop_norm = o.stop_norm;
    c->inA.tol = o.tol_inner_A;
    c->inA.max_iter = o.max_inner;
    c->rec.tol = o.tol_inner_A;
    c->rec.max_iter = o.max_inner;
    c->inS.tol = o.tol_inner_S;
    c->inS.max_iter = o.max_inner;
    c->out.tol = o.tol;
    c->out.max_iter = o.max_outer;
    c->inA32.tol = o.tol_inner_f32;
    c->inA32.max_iter = o.max_inner;
    c->inS32.tol = o.tol_inner_f32;
    c->inS32.max_iter = o.max_inner;
    c->mix.max_refine = o.max_refine;
    c->mix.step_max = o.step_max;
    c->mix.factor = o.refine_factor;
    c->mix.refine = 0;
    c->mix.stop = 0;
    c->zero_rhs = 0;
    H.last_loop = o.loop_mode;
    H.last_precision = o.precision;
    return SCHUR_OK;
}

int upload_ctl(Handle& H) { return upload(H); }

int download_ctl_async(Handle& H) {
    CUDA_TRY(cudaMemcpyAsync(H.hctl, H.dctl, sizeof(Ctl), cudaMemcpyDeviceToHost, H.stream),
             "control download");
    return SCHUR_OK;
}

void fill_solve_stats(Handle& H, int precision, schur_stats* stats) {
    const Ctl* c = H.hctl;
    std::memset(stats, 0, sizeof(*stats));
    stats->status = call_status(c, c->out.status);
    stats->outer_iters = c->out.iter;
    stats->zero_rhs = c->zero_rhs;
    stats->inner_status = map_status(c->inner_status);
    stats->inner_iters_A = c->inA.total;
    stats->inner_iters_S = c->inS.total;
    stats->rel_res = c->out.rel;
    stats->rel_res_precond = c->out.relz;
    stats->g_norm = std::sqrt(c->g_norm2);
    stats->kernel_launches = c->launches;
    stats->inner_iters_A_f32 = c->inA32.total;
    stats->inner_iters_S_f32 = c->inS32.total;
    stats->refinements = precision == SCHUR_MIXED ? c->mix.refine : 0;
}

void fill_recover_stats(Handle& H, schur_stats* stats) {
    const Ctl* c = H.hctl;
    std::memset(stats, 0, sizeof(*stats));
    stats->status = call_status(c, c->rec.status);
    stats->inner_status = map_status(c->inner_status);
    stats->inner_iters_A = c->rec.total;
    stats->rel_res = c->rec.rel;
    stats->kernel_launches = c->launches;
}

}  // namespace schur

extern "C" {

void schur_opts_default(schur_opts* o) {
    if (!o) return;
    o->precond = SCHUR_SIMPLE;
    o->stop_norm = SCHUR_STOP_UNPRECOND;
    o->precision = SCHUR_FP64;
    o->loop_mode = SCHUR_LOOP_GRAPH;
    o->max_outer = 2000;
    o->max_inner = 20000;
    o->tol = 1e-8;
    o->tol_inner_A = 1e-12;
    o->tol_inner_S = 1e-12;
    o->tol_inner_f32 = 1e-4;
    o->refine_factor = 1e-3;
    o->max_refine = 30;
    o->step_max = 1000;
    o->inner_precond = SCHUR_INNER_JACOBI;
}

const char* schur_last_error(void) { return g_last_error.c_str(); }

int schur_create_geometry(const uint8_t* mask, int ndim, const int64_t dims[3],
                          const int periodic[3], void* stream, schur_geom_t* out) {
    NvtxRange nvtx_("schur_create_geometry");
    if (!out) return set_error(SCHUR_EINVAL, "out is NULL");
    *out = nullptr;
    if (!mask || !dims || !periodic) return set_error(SCHUR_EINVAL, "mask, dims or periodic is NULL");
    if (ndim != 2 && ndim != 3) return set_error(SCHUR_EINVAL, "ndim must be 2 or 3");
    for (int a = 0; a < ndim; ++a)
        if (dims[a] < 2 || dims[a] > (1 << 20))
            return set_error(SCHUR_EINVAL, "every extent must lie in [2, 2^20]");
    const long long nz = ndim == 3 ? dims[2] : 1;
    const long long ncell = dims[0] * dims[1] * nz;
    if (ncell > 1400000000ll)  // 32-bit work-list entries over [d][stride]
        return set_error(SCHUR_EINVAL, "grid too large (more than 1.4e9 cells)");

    schur_geom* G = new schur_geom();
    Handle& H = G->H;
    H.stream = (cudaStream_t)stream;
    Dev& g = H.g;
    g.nx = (int)dims[0];
    g.ny = (int)dims[1];
    g.nz = (int)nz;
    g.d = ndim;
    g.per[0] = periodic[0] != 0;
    g.per[1] = periodic[1] != 0;
    g.per[2] = ndim == 3 ? periodic[2] != 0 : 1;
    g.ncell = ncell;
    g.stride = round_up(ncell, 64);
    g.h = 1.0 / (double)g.nx;
    g.hinv = (double)g.nx;
    g.h2 = g.h * g.h;
    g.h2inv = g.hinv * g.hinv;
    for (int k = 0; k < 5; ++k) {
        g.diag[k] = (double)(2 * ndim + k);
        g.wdiag[k] = 1.0 / g.diag[k];
        g.diagf[k] = (float)g.diag[k];
        g.wdiagf[k] = (float)g.wdiag[k];
    }

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&H.nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        delete G;
        return cuda_error(e, "device query");
    }
    H.target_blocks = H.nsm * 8 < kMaxBlocks ? H.nsm * 8 : kMaxBlocks;

    const size_t nf = (size_t)g.d * g.stride;
    const size_t nc = (size_t)ncell;
    cudaError_t ea = cudaSuccess;
    auto A = [&](auto** p, size_t n) { if (ea == cudaSuccess) ea = alloc(H, p, n); };
    A(&H.mask, nc);
    A(&H.flags, nf);
    A(&H.invdS, nc);
    A(&H.op, nc); A(&H.orr, nc); A(&H.od, nc); A(&H.oq, nc); A(&H.og, nc);
    A(&H.u, nf);
    A(&H.partials, (size_t)kMaxBlocks * 8);
    A(&H.dctl, 1);
    if (ea == cudaSuccess) ea = cudaMallocHost((void**)&H.hctl, sizeof(Ctl));
    if (ea != cudaSuccess) {
        free_all(H);
        delete G;
        if (ea == cudaErrorMemoryAllocation)
            return set_error(SCHUR_ENOMEM, "device allocation failed");
        return cuda_error(ea, "allocation");
    }
    std::memset(H.hctl, 0, sizeof(Ctl));

    // mask: host or device pointer
    cudaPointerAttributes attr;
    cudaMemcpyKind kind = cudaMemcpyHostToDevice;
    if (cudaPointerGetAttributes(&attr, mask) == cudaSuccess &&
        (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged))
        kind = cudaMemcpyDeviceToDevice;
    cudaGetLastError();
    e = cudaMemcpyAsync(H.mask, mask, nc, kind, H.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(H.dctl, H.hctl, sizeof(Ctl), cudaMemcpyHostToDevice, H.stream);
    if (e == cudaSuccess) e = launch_flags(H);
    if (e == cudaSuccess) e = launch_invdiag_simple(H);
    if (e == cudaSuccess) e = cudaMemcpyAsync(H.hctl, H.dctl, sizeof(Ctl), cudaMemcpyDeviceToHost, H.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(H.stream);
    if (e != cudaSuccess) {
        int rc = cuda_error(e, "geometry build");
        free_all(H);
        delete G;
        return rc;
    }
    if (H.hctl->counts[4] != 0.0) {
        free_all(H);
        delete G;
        return set_error(SCHUR_EINVAL, "mask values must be 0 (solid) or 1 (fluid)");
    }
    // components are labelled on the host
    std::vector<uint8_t> hmask;
    const uint8_t* hm = mask;
    if (kind == cudaMemcpyDeviceToDevice) {
        hmask.resize(nc);
        e = cudaMemcpy(hmask.data(), H.mask, nc, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            int rc = cuda_error(e, "mask download");
            free_all(H);
            delete G;
            return rc;
        }
        hm = hmask.data();
    }
    int rc = build_components(H, hm);
    if (rc == SCHUR_OK) rc = upload(H);
    if (rc == SCHUR_OK) {
        e = cudaStreamSynchronize(H.stream);
        if (e != cudaSuccess) rc = cuda_error(e, "geometry build");
    }
    if (rc != SCHUR_OK) {
        free_all(H);
        delete G;
        return rc;
    }
    *out = G;
    return SCHUR_OK;
}

int schur_set_force(schur_geom_t G, const double f[3]) {
    if (!G || !f) return set_error(SCHUR_EINVAL, "null argument");
    for (int a = 0; a < 3; ++a) {
        if (!std::isfinite(f[a])) return set_error(SCHUR_EINVAL, "force must be finite");
        G->H.force[a] = (a < G->H.g.d) ? f[a] : 0.0;
    }
    G->H.solved = G->H.recovered = false;
    return SCHUR_OK;
}

int schur_solve(schur_geom_t G, const schur_opts* opts, schur_stats* stats) {
    NvtxRange nvtx_("schur_solve");
    if (!G) return set_error(SCHUR_EINVAL, "null handle");
    schur_opts o;
    if (opts) o = *opts; else schur_opts_default(&o);
    Handle& H = G->H;
    if (H.pending) return set_error(SCHUR_ESTATE, "an asynchronous solve is in flight");
    int rc = check_opts(o);
    if (rc) return rc;
    o = resolve_precond(H, o);
    if ((rc = prepare_solve(H, o, o.loop_mode == SCHUR_LOOP_GRAPH))) return rc;
    const int gi = o.precision * 2 + o.precond;
    if (o.loop_mode == SCHUR_LOOP_GRAPH) {
        rc = build_graph(H, &H.graph_solve[gi], &H.exec_solve[gi],
                         [&](Recorder& R) { record_solve(H, R, o.precond, o.precision); });
        if (rc) return rc;
        if ((rc = upload(H))) return rc;
        CUDA_TRY(cudaGraphLaunch(H.exec_solve[gi], H.stream), "cudaGraphLaunch");
    } else {
        if ((rc = upload(H))) return rc;
        int slot = kHostSlotBase;
        Recorder R(H.stream, H.dctl, &slot);
        record_solve(H, R, o.precond, o.precision);
        if (!R.ok()) return cuda_error(R.error(), R.where().c_str());
    }
    if ((rc = download(H))) return rc;
    H.solved = true;
    H.recovered = false;
    if (stats) fill_solve_stats(H, o.precision, stats);
    const int st = call_status(H.hctl, H.hctl->out.status);
    if (st != SCHUR_OK) set_error(st, status_text(H, "outer iteration did not converge"));
    return st;
}

int schur_recover_velocity(schur_geom_t G, schur_stats* stats) {
    NvtxRange nvtx_("schur_recover_velocity");
    if (!G) return set_error(SCHUR_EINVAL, "null handle");
    Handle& H = G->H;
    if (H.pending) return set_error(SCHUR_ESTATE, "an asynchronous solve is in flight");
    if (!H.solved) return set_error(SCHUR_ESTATE, "recover_velocity needs a schur_solve first");
    reset_call(H, H.last_loop == SCHUR_LOOP_GRAPH);
    int rc;
    if (H.last_loop == SCHUR_LOOP_GRAPH) {
        rc = build_graph(H, &H.graph_recover, &H.exec_recover,
                         [&](Recorder& R) { record_recover(H, R); });
        if (rc) return rc;
        if ((rc = upload(H))) return rc;
        CUDA_TRY(cudaGraphLaunch(H.exec_recover, H.stream), "cudaGraphLaunch");
    } else {
        if ((rc = upload(H))) return rc;
        int slot = kHostSlotBase;
        Recorder R(H.stream, H.dctl, &slot);
        record_recover(H, R);
        if (!R.ok()) return cuda_error(R.error(), R.where().c_str());
    }
    if ((rc = download(H))) return rc;
    H.recovered = true;
    if (stats) fill_recover_stats(H, stats);
    const int st = call_status(H.hctl, H.hctl->rec.status);
    if (st != SCHUR_OK) set_error(st, status_text(H, "velocity recovery did not converge"));
    return st;
}

int schur_solve_async(schur_geom_t G, const schur_opts* opts) {
    NvtxRange nvtx_("schur_solve_async");
    if (!G) return set_error(SCHUR_EINVAL, "null handle");
    schur_opts o;
    if (opts) o = *opts; else schur_opts_default(&o);
    o.loop_mode = SCHUR_LOOP_GRAPH;
    Handle& H = G->H;
    if (H.pending) return set_error(SCHUR_ESTATE, "an asynchronous solve is in flight");
    int rc = check_opts(o);
    if (rc) return rc;
    o = resolve_precond(H, o);
    if ((rc = prepare_solve(H, o, 1))) return rc;
    const int gi = o.precision * 2 + o.precond;
    rc = build_graph(H, &H.graph_full[gi], &H.exec_full[gi],
                     [&](Recorder& R) { record_solve_recover(H, R, o.precond, o.precision); });
    if (rc) return rc;
    if (!H.done_ev) CUDA_TRY(cudaEventCreateWithFlags(&H.done_ev, cudaEventDisableTiming), "event");
    if ((rc = upload(H))) return rc;
    CUDA_TRY(cudaGraphLaunch(H.exec_full[gi], H.stream), "cudaGraphLaunch");
    if ((rc = download_ctl_async(H))) return rc;
    CUDA_TRY(cudaEventRecord(H.done_ev, H.stream), "event record");
    H.pending = true;
    H.pending_precision = o.precision;
    H.solved = H.recovered = false;
    return SCHUR_OK;
}

int schur_query(schur_geom_t G, int* done) {
    if (!G || !done) return set_error(SCHUR_EINVAL, "null argument");
    Handle& H = G->H;
    if (!H.pending) { *done = 1; return SCHUR_OK; }
    cudaError_t e = cudaEventQuery(H.done_ev);
    if (e == cudaErrorNotReady) { *done = 0; return SCHUR_OK; }
    if (e != cudaSuccess) return cuda_error(e, "event query");
    *done = 1;
    return SCHUR_OK;
}

int schur_finish(schur_geom_t G, schur_stats* solve_stats, schur_stats* recover_stats) {
    if (!G) return set_error(SCHUR_EINVAL, "null handle");
    Handle& H = G->H;
    if (!H.pending) return set_error(SCHUR_ESTATE, "no asynchronous solve in flight");
    CUDA_TRY(cudaEventSynchronize(H.done_ev), "event synchronize");
    H.pending = false;
    H.solved = H.recovered = true;
    if (solve_stats) fill_solve_stats(H, H.pending_precision, solve_stats);
    if (recover_stats) fill_recover_stats(H, recover_stats);
    int st = call_status(H.hctl, H.hctl->out.status);
    if (st == SCHUR_OK) st = call_status(H.hctl, H.hctl->rec.status);
    if (st != SCHUR_OK) set_error(st, status_text(H, "solve or recovery did not converge"));
    return st;
}

int schur_permeability(schur_geom_t G, int axis, double* k_out) {
    if (!G || !k_out) return set_error(SCHUR_EINVAL, "null argument");
    Handle& H = G->H;
    if (axis < 0 || axis >= H.g.d) return set_error(SCHUR_EINVAL, "axis out of range");
    if (!H.recovered) return set_error(SCHUR_ESTATE, "permeability needs recover_velocity first");
    *k_out = H.hctl->perm[axis];
    return SCHUR_OK;
}

int schur_permeability_diag(schur_geom_t G, const schur_opts* opts, double k_out[3],
                            schur_stats* stats) {
    NvtxRange nvtx_("schur_permeability_diag");
    if (!G || !k_out) return set_error(SCHUR_EINVAL, "null argument");
    Handle& H = G->H;
    if (H.pending) return set_error(SCHUR_ESTATE, "an asynchronous solve is in flight");
    int worst = SCHUR_OK;
    std::string msg;
    for (int a = 0; a < 3; ++a) k_out[a] = 0.0;
    for (int a = 0; a < H.g.d; ++a) {
        double f[3] = {0.0, 0.0, 0.0};
        f[a] = 1.0;
        int rc = schur_set_force(G, f);
        if (rc == SCHUR_OK || rc == SCHUR_ENOTCONV) {
            rc = schur_solve(G, opts, stats ? &stats[a] : nullptr);
            if (rc == SCHUR_OK || rc == SCHUR_ENOTCONV) {
                const int rr = schur_recover_velocity(G, nullptr);
                if (rr != SCHUR_OK && rc == SCHUR_OK) rc = rr;
                if (H.recovered) k_out[a] = H.hctl->perm[a];
            }
        }
        if (rc != SCHUR_OK) {
            if (worst == SCHUR_OK || rc == SCHUR_ECUDA || rc == SCHUR_ENOMEM) {
                worst = rc;
                msg = schur_last_error();
            }
            if (rc != SCHUR_ENOTCONV && rc != SCHUR_EBREAKDOWN) break;
        }
    }
    if (worst != SCHUR_OK) set_error(worst, msg.c_str());
    return worst;
}

int schur_history(schur_geom_t G, int cap, double* alpha, double* beta, double* rel,
                  double* relz, int* n) {
    if (!G || !n || cap < 0) return set_error(SCHUR_EINVAL, "bad history arguments");
    Handle& H = G->H;
    if (H.pending) return set_error(SCHUR_ESTATE, "an asynchronous solve is in flight");
    if (!H.solved) return set_error(SCHUR_ESTATE, "history needs a schur_solve first");
    const int m = std::min({H.hctl->out.iter, H.hist_cap, cap});
    *n = std::min(H.hctl->out.iter, H.hist_cap);
    if (m <= 0) return SCHUR_OK;
    std::vector<double> h((size_t)m * 4);
    CUDA_TRY(cudaMemcpyAsync(h.data(), H.hist, h.size() * sizeof(double), cudaMemcpyDeviceToHost,
                             H.stream), "history download");
    CUDA_TRY(cudaStreamSynchronize(H.stream), "stream synchronize");
    for (int k = 0; k < m; ++k) {
        if (alpha) alpha[k] = h[4 * k + 0];
        if (beta) beta[k] = h[4 * k + 1];
        if (rel) rel[k] = h[4 * k + 2];
        if (relz) relz[k] = h[4 * k + 3];
    }
    return SCHUR_OK;
}

int schur_lanczos_extremes(const double* alpha, const double* beta, int m, double* lmin,
                           double* lmax) {
    if (!alpha || (m > 1 && !beta) || !lmin || !lmax || m < 1)
        return set_error(SCHUR_EINVAL, "bad Lanczos arguments");
    // Lanczos tridiagonal of CG (Saad, Section 6.7.3): T[j][j] = 1/a_j + b_(j-1)/a_(j-1),
    // T[j][j+1] = sqrt(b_j)/a_j
    std::vector<double> d(m), e(m > 1 ? m - 1 : 0);
    for (int j = 0; j < m; ++j) {
        if (!(alpha[j] > 0.0) || (j + 1 < m && !(beta[j] >= 0.0)))
            return set_error(SCHUR_EINVAL, "CG coefficients must be alpha > 0, beta >= 0");
        d[j] = 1.0 / alpha[j] + (j ? beta[j - 1] / alpha[j - 1] : 0.0);
        if (j + 1 < m) e[j] = std::sqrt(beta[j]) / alpha[j];
    }
    *lmin = tridiag_eig(d, e, 0);
    *lmax = tridiag_eig(d, e, m - 1);
    return SCHUR_OK;
}

int schur_cond_estimate(schur_geom_t G, double* lmin, double* lmax, double* cond) {
    if (!G || !lmin || !lmax || !cond) return set_error(SCHUR_EINVAL, "null argument");
    Handle& H = G->H;
    if (H.pending) return set_error(SCHUR_ESTATE, "an asynchronous solve is in flight");
    if (!H.solved || H.last_precision != SCHUR_FP64)
        return set_error(SCHUR_ESTATE, "the estimate needs the coefficients of an FP64 solve "
                                       "(flexible CG coefficients define no Lanczos matrix)");
    const int m = std::min(H.hctl->out.iter, H.hist_cap);
    if (m < 1) return set_error(SCHUR_ESTATE, "the last solve made no outer iteration");
    std::vector<double> a(m), b(m);
    int n = 0;
    int rc = schur_history(G, m, a.data(), b.data(), nullptr, nullptr, &n);
    if (rc) return rc;
    rc = schur_lanczos_extremes(a.data(), b.data(), m, lmin, lmax);
    if (rc) return set_error(SCHUR_ESTATE, "the recorded CG coefficients are not usable");
    *cond = *lmax / *lmin;
    return SCHUR_OK;
}

int schur_get_field(schur_geom_t G, int which, void** dev_ptr, int64_t* elems, int* dtype) {
    if (!G || !dev_ptr) return set_error(SCHUR_EINVAL, "null argument");
    Handle& H = G->H;
    const int64_t nf = (int64_t)H.g.d * H.g.stride, nc = H.g.ncell;
    void* p = nullptr;
    int64_t n = 0;
    int dt = 0;
    switch (which) {
        case SCHUR_FIELD_P: p = H.op; n = nc; dt = SCHUR_DTYPE_F64; break;
        case SCHUR_FIELD_U: p = H.u; n = nf; dt = SCHUR_DTYPE_F64; break;
        case SCHUR_FIELD_FLAGS: p = H.flags; n = nf; dt = SCHUR_DTYPE_U8; break;
        case SCHUR_FIELD_MASK: p = H.mask; n = nc; dt = SCHUR_DTYPE_U8; break;
        case SCHUR_FIELD_G: p = H.og; n = nc; dt = SCHUR_DTYPE_F64; break;
        default: return set_error(SCHUR_EINVAL, "unknown field");
    }
    *dev_ptr = p;
    if (elems) *elems = n;
    if (dtype) *dtype = dt;
    return SCHUR_OK;
}

int schur_geometry_info(schur_geom_t G, schur_geom_info* info) {
    if (!G || !info) return set_error(SCHUR_EINVAL, "null argument");
    Handle& H = G->H;
    std::memset(info, 0, sizeof(*info));
    info->ndim = H.g.d;
    info->dims[0] = H.g.nx;
    info->dims[1] = H.g.ny;
    info->dims[2] = H.g.d == 3 ? H.g.nz : 1;
    for (int a = 0; a < 3; ++a) info->periodic[a] = H.g.per[a];
    info->n_cells = H.g.ncell;
    info->face_stride = H.g.stride;
    for (int a = 0; a < 3; ++a) info->n_unknown[a] = (int64_t)H.hctl->counts[a];
    info->n_fluid = (int64_t)H.hctl->counts[3];
    info->h = H.g.h;
    info->device_bytes = H.bytes;
    return SCHUR_OK;
}

int schur_apply_A(schur_geom_t G, const double* x, double* y) {
    if (!G || !x || !y) return set_error(SCHUR_EINVAL, "null argument");
    cudaError_t e = launch_apply_A(G->H, x, y);
    return e == cudaSuccess ? SCHUR_OK : cuda_error(e, "apply_A");
}

int schur_apply_B(schur_geom_t G, const double* u, double* p) {
    if (!G || !u || !p) return set_error(SCHUR_EINVAL, "null argument");
    cudaError_t e = launch_apply_B(G->H, u, p);
    return e == cudaSuccess ? SCHUR_OK : cuda_error(e, "apply_B");
}

int schur_apply_BT(schur_geom_t G, const double* p, double* u) {
    if (!G || !p || !u) return set_error(SCHUR_EINVAL, "null argument");
    cudaError_t e = launch_apply_BT(G->H, p, u);
    return e == cudaSuccess ? SCHUR_OK : cuda_error(e, "apply_BT");
}

int schur_apply_simple(schur_geom_t G, const double* p, double* q) {
    if (!G || !p || !q) return set_error(SCHUR_EINVAL, "null argument");
    cudaError_t e = launch_apply_simple(G->H, p, q);
    return e == cudaSuccess ? SCHUR_OK : cuda_error(e, "apply_simple");
}

int schur_solve_A(schur_geom_t G, const double* b, double* x, double tol, int max_iter,
                  int* iters) {
    NvtxRange nvtx_("schur_solve_A");
    if (!G || !b || !x) return set_error(SCHUR_EINVAL, "null argument");
    if (!(tol > 0) || max_iter < 1) return set_error(SCHUR_EINVAL, "tol must be > 0, max_iter >= 1");
    Handle& H = G->H;
    const size_t nf = (size_t)H.g.d * H.g.stride;
    Ctl* c = H.hctl;
    reset_call(H, 1);
    c->solo.tol = tol;
    c->solo.max_iter = max_iter;
    // the right-hand side is staged in a dense buffer of the handle (allocated on first use)
    if (!H.stage) {
        cudaError_t e = alloc(H, &H.stage, nf);
        if (e == cudaErrorMemoryAllocation) return set_error(SCHUR_ENOMEM, "device allocation failed");
        if (e != cudaSuccess) return cuda_error(e, "staging buffer");
    }
    CUDA_TRY(cudaMemcpyAsync(H.stage, b, nf * sizeof(double), cudaMemcpyDeviceToDevice, H.stream),
             "stage rhs");
    int rc = build_graph(H, &H.graph_solo, &H.exec_solo,
                         [&](Recorder& R) { record_solve_A(H, R, H.stage, H.ax); });
    if (rc) return rc;
    if ((rc = upload(H))) return rc;
    CUDA_TRY(cudaGraphLaunch(H.exec_solo, H.stream), "cudaGraphLaunch");
    CUDA_TRY(cudaMemsetAsync(x, 0, nf * sizeof(double), H.stream), "clear solution");
    CUDA_TRY(launch_scatter_f64(H, H.ax, H.ulist, x, H.n_u), "scatter solution");
    if ((rc = download(H))) return rc;
    if (iters) *iters = c->solo.iter;
    const int st = call_status(c, c->solo.status);
    if (st != SCHUR_OK) set_error(st, status_text(H, "inner A solve did not converge"));
    return st;
}

int schur_set_launch(schur_geom_t G, int blocks_per_sm, int entries_per_thread,
                     int persistent_inner) {
    if (!G) return set_error(SCHUR_EINVAL, "null handle");
    return set_launch_shape(G->H, blocks_per_sm, entries_per_thread, persistent_inner);
}

int schur_set_barrier_limit(schur_geom_t G, unsigned int polls, int skip_block) {
    if (!G) return set_error(SCHUR_EINVAL, "null handle");
    if (skip_block < -1 || skip_block >= kMaxBlocks)
        return set_error(SCHUR_EINVAL, "skip_block must be -1 or a block index below 4096");
    Handle& H = G->H;
    if (H.pending) return set_error(SCHUR_ESTATE, "an asynchronous solve is in flight");
    H.hctl->bar_limit = polls;
    H.hctl->bar_skip = skip_block + 1;
    return SCHUR_OK;
}

int schur_time_kernel(schur_geom_t G, int kernel, float* ms) {
    if (!G || !ms) return set_error(SCHUR_EINVAL, "null argument");
    if (kernel < 0 || kernel > 19) return set_error(SCHUR_EINVAL, "kernel id must be 0..19");
    if (((kernel > 5 && kernel < 12) || kernel == 14 || kernel == 15 || kernel > 17) && !G->H.axf)
        return set_error(SCHUR_ESTATE, "FP32 kernels need a mixed-precision solve first");
    Handle& H = G->H;
    if (kernel >= 16 && !((kernel & 1) ? H.mgS.nlev : H.mgA.nlev))
        return set_error(SCHUR_ESTATE, "multigrid kernels need a solve with SCHUR_INNER_MG first");
    reset_call(H, 0);  // no graph: the condition slot is only written to device memory
    int rc = upload(H);
    if (rc) return rc;
    cudaError_t e = time_kernel(H, kernel, kSlots - 1, ms);
    if (e != cudaSuccess) return cuda_error(e, "time_kernel");
    return download(H);
}

int schur_mg_levels(schur_geom_t G, int simple, int64_t* sizes, int max_levels, int* nlev,
                    int* tail) {
    if (!G || !nlev || !tail || (sizes && max_levels < 0))
        return set_error(SCHUR_EINVAL, "null or bad argument");
    const MgOp& M = simple ? G->H.mgS : G->H.mgA;
    *nlev = M.nlev;
    *tail = M.tail;
    if (sizes)
        for (int l = 0; l < M.nlev && l < max_levels; ++l) sizes[l] = (int64_t)M.n[l];
    return SCHUR_OK;
}

int schur_fp64_peak(void* stream, int iters, double* lane_ops_per_s) {
    if (!lane_ops_per_s) return set_error(SCHUR_EINVAL, "null argument");
    if (iters < 1 || iters > (1 << 20)) return set_error(SCHUR_EINVAL, "iters must lie in [1, 2^20]");
    cudaError_t e = measure_fp64_peak((cudaStream_t)stream, iters, lane_ops_per_s);
    if (e != cudaSuccess) return cuda_error(e, "fp64 peak");
    return SCHUR_OK;
}

void schur_destroy(schur_geom_t G) {
    if (!G) return;
    cudaStreamSynchronize(G->H.stream);
    free_all(G->H);
    delete G;
}

}  // extern "C"
