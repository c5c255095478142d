// Batched and served execution of many geometries on one GPU.
//
// Batch: the solve + recovery control flow of every geometry is recorded as one branch
// of a single CUDA graph (each branch with its own conditional loops, control block and
// reduction scratch), so one cudaGraphLaunch runs all of them and the GPU overlaps the
// branches.  The launch shape of every branch (blocks per SM of its kernels) is a free
// parameter; schur_batch_autotune times the whole batch for a few candidates.
//
// Server: a request loop driven by the caller.  Submitted jobs wait in FIFO order and
// are admitted while their estimated device footprint fits the memory budget and the
// number of running jobs is below the cap; each admitted job gets its own stream,
// geometry and one graph launch (solve + recovery), so jobs that arrive while others
// run start as soon as memory frees up and their work overlaps on the device.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <string>
#include <vector>

#include "internal.h"

using namespace schur;

// Geometries that share the GPU (batch branches, served jobs) size their grids by work as
// well: at least this many entries per thread, so that a small geometry takes a few SMs
// and leaves the rest to the others (the inner loop kernels hold their SMs for a whole
// inner solve).
constexpr int kSharedEntriesPerThread = 16;

// ------------------------------------------------------------------------------------
// batch
// ------------------------------------------------------------------------------------


struct schur_batch {
    std::vector<schur_geom_t> geoms;
    schur_opts opts{};
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int blocks_per_sm = 8;
};

static void batch_free(schur_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

extern "C" int schur_batch_create(schur_geom_t* geoms, int n, const schur_opts* opts,
                                  int blocks_per_sm, void* stream, schur_batch_t* out) {
    if (!geoms || n < 1 || !out) return schur_set_error_internal(SCHUR_EINVAL, "bad batch arguments");
    *out = nullptr;
    schur_opts o;
    if (opts) o = *opts; else schur_opts_default(&o);
    o.loop_mode = SCHUR_LOOP_GRAPH;
    int rc = check_opts(o);
    if (rc) return rc;
    if (blocks_per_sm < 0 || blocks_per_sm > 32)
        return schur_set_error_internal(SCHUR_EINVAL, "blocks_per_sm must lie in [0, 32]");
    schur_batch* b = new schur_batch();
    b->geoms.assign(geoms, geoms + n);
    b->opts = o;
    b->stream = (cudaStream_t)stream;
    b->blocks_per_sm = blocks_per_sm;
    cudaError_t e = cudaGraphCreate(&b->graph, 0);
    if (e != cudaSuccess) {
        delete b;
        return schur_set_error_internal(SCHUR_ECUDA, cudaGetErrorString(e));
    }
    for (int i = 0; i < n; ++i) {
        if (!geoms[i]) {
            batch_free(b);
            delete b;
            return schur_set_error_internal(SCHUR_EINVAL, "null geometry in batch");
        }
        Handle& H = handle_of(geoms[i]);
        if (H.pending) {
            batch_free(b);
            delete b;
            return schur_set_error_internal(SCHUR_ESTATE, "a geometry has an asynchronous solve in flight");
        }
        if ((blocks_per_sm > 0 &&
             (rc = set_launch_shape(H, blocks_per_sm, kSharedEntriesPerThread, 1))) ||
            (rc = prepare_solve(H, resolve_precond(H, o), 1))) {
            batch_free(b);
            delete b;
            return rc;
        }
        const size_t before = H.handles.size();
        Recorder R(b->graph, H.dctl, &H.next_slot, &H.handles);  // branch from the graph root
        record_solve_recover(H, R, resolve_precond(H, o).precond, o.precision);
        if (!R.ok()) {
            std::string msg = "batch recording: " + R.where();
            batch_free(b);
            delete b;
            return schur_set_error_internal(SCHUR_ECUDA, msg.c_str());
        }
        for (size_t k = before; k < H.handles.size(); ++k)
            H.hctl->handle[H.handles[k].first] = H.handles[k].second;
    }
    e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) {
        batch_free(b);
        delete b;
        return schur_set_error_internal(SCHUR_ECUDA, cudaGetErrorString(e));
    }
    *out = b;
    return SCHUR_OK;
}

// One launch of the batch graph.  stats arrays (may be NULL) have n entries; k_out (may
// be NULL) receives 3 permeabilities per geometry.
extern "C" int schur_batch_run(schur_batch_t b, schur_stats* solve_stats,
                               schur_stats* recover_stats, double* k_out) {
    NvtxRange nvtx_("schur_batch_run");
    if (!b) return schur_set_error_internal(SCHUR_EINVAL, "null batch");
    int rc;
    for (schur_geom_t g : b->geoms) {
        Handle& H = handle_of(g);
        if ((rc = prepare_solve(H, b->opts, 1))) return rc;
        // the batch runs on its own stream: stage the control block there
        cudaError_t e = cudaMemcpyAsync(H.dctl, H.hctl, sizeof(Ctl), cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) return schur_set_error_internal(SCHUR_ECUDA, cudaGetErrorString(e));
    }
    cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
    if (e != cudaSuccess) return schur_set_error_internal(SCHUR_ECUDA, cudaGetErrorString(e));
    for (schur_geom_t g : b->geoms) {
        Handle& H = handle_of(g);
        e = cudaMemcpyAsync(H.hctl, H.dctl, sizeof(Ctl), cudaMemcpyDeviceToHost, b->stream);
        if (e != cudaSuccess) return schur_set_error_internal(SCHUR_ECUDA, cudaGetErrorString(e));
    }
    e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return schur_set_error_internal(SCHUR_ECUDA, cudaGetErrorString(e));
    int worst = SCHUR_OK;
    for (size_t i = 0; i < b->geoms.size(); ++i) {
        Handle& H = handle_of(b->geoms[i]);
        H.solved = H.recovered = true;
        if (solve_stats) fill_solve_stats(H, b->opts.precision, &solve_stats[i]);
        if (recover_stats) fill_recover_stats(H, &recover_stats[i]);
        if (k_out)
            for (int a = 0; a < 3; ++a) k_out[3 * i + a] = H.hctl->perm[a];
        const int s1 = H.hctl->out.status, s2 = H.hctl->rec.status;
        if (H.hctl->bar_err) worst = SCHUR_ECUDA;
        else if (worst == SCHUR_ECUDA) continue;
        else if (s1 == ST_BREAKDOWN || s2 == ST_BREAKDOWN) worst = SCHUR_EBREAKDOWN;
        else if ((s1 != ST_OK || s2 != ST_OK) && worst == SCHUR_OK) worst = SCHUR_ENOTCONV;
    }
    if (worst != SCHUR_OK) schur_set_error_internal(worst, "a batch member did not converge");
    return worst;
}

extern "C" void schur_batch_destroy(schur_batch_t b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_free(b);
    delete b;
}

// Launch shapes tried by the autotuner: {blocks_per_sm, entries_per_thread, persistent}.
// Persistent inner loops make each solve faster but hold their SMs for a whole inner
// solve; per-phase graph nodes let many geometries interleave.
static const int kTuneShapes[][3] = {
    {8, 1, 0}, {2, 1, 0}, {8, kSharedEntriesPerThread, 1}, {2, kSharedEntriesPerThread, 1},
    {1, kSharedEntriesPerThread, 1}};

// Time the whole batch for every shape of kTuneShapes (one untimed and one timed run
// each) and keep the fastest on the geometries.
extern "C" int schur_batch_autotune(schur_geom_t* geoms, int n, const schur_opts* opts,
                                    void* stream, int best_shape[3], double* best_ms) {
    if (!best_shape || !geoms || n < 1)
        return schur_set_error_internal(SCHUR_EINVAL, "bad autotune arguments");
    double best = 1e300;
    int arg = 0;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return schur_set_error_internal(SCHUR_ECUDA, "event create");
    const int nshape = (int)(sizeof(kTuneShapes) / sizeof(kTuneShapes[0]));
    int rc = SCHUR_OK;
    for (int c = 0; c < nshape && rc == SCHUR_OK; ++c) {
        const int* sh = kTuneShapes[c];
        for (int i = 0; i < n && rc == SCHUR_OK; ++i)
            rc = set_launch_shape(handle_of(geoms[i]), sh[0], sh[1], sh[2]);
        schur_batch_t b = nullptr;
        if (rc == SCHUR_OK) rc = schur_batch_create(geoms, n, opts, 0, stream, &b);
        if (rc != SCHUR_OK) break;
        schur_batch_run(b, nullptr, nullptr, nullptr);  // warm-up
        cudaEventRecord(e0, (cudaStream_t)stream);
        const int rr = schur_batch_run(b, nullptr, nullptr, nullptr);
        cudaEventRecord(e1, (cudaStream_t)stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        schur_batch_destroy(b);
        if (rr == SCHUR_OK && ms < best) {
            best = ms;
            arg = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != SCHUR_OK) return rc;
    const int* sh = kTuneShapes[arg];
    for (int i = 0; i < n; ++i) set_launch_shape(handle_of(geoms[i]), sh[0], sh[1], sh[2]);
    for (int k = 0; k < 3; ++k) best_shape[k] = sh[k];
    if (best_ms) *best_ms = best;
    return SCHUR_OK;
}

// ------------------------------------------------------------------------------------
// server
// ------------------------------------------------------------------------------------

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    int64_t id;
    std::vector<uint8_t> mask;
    int ndim;
    int64_t dims[3];
    int periodic[3];
    int axis;
    int precond = SCHUR_UZAWA;
    int64_t bytes;
    double t_submit, t_start = 0, t_done = 0;
    schur_geom_t geom = nullptr;
    cudaStream_t stream = nullptr;
};

}  // namespace

struct schur_server {
    schur_opts opts{};
    int64_t budget = 0;
    int max_active = 1;
    int64_t used = 0;
    int64_t next_id = 1;
    Clock::time_point t0;
    std::deque<Job> pending;
    std::vector<Job> active;
    std::vector<schur_job_result> done;
    int64_t peak_used = 0;
    int peak_active = 0;
    // launch shape of every job: per-phase graph nodes, so that the jobs in flight
    // interleave at phase granularity (measured: higher capacity than persistent loops)
    int shape[3] = {8, 1, 0};
};

static double now_s(const schur_server* s) {
    return std::chrono::duration<double>(Clock::now() - s->t0).count();
}

// Device bytes of one job, an upper bound from the allocations schur_create_geometry and
// a solve make, counting every face as an unknown and every cell as fluid.  Per face
// (d x cells): flags 1, velocity 8, work list 4, flag copy 1, four FP64 inner vectors 32,
// neighbour table 8d (2d 4-byte entries).  Per cell: mask 1, S-hat inverse diagonal
// (dense and compact) and diagonal 24, component id 4, cell list 4, five outer and four
// SIMPLE FP64 vectors 72, neighbour table 8d, face codes 4.  Mixed precision adds four
// FP32 vectors per face and five per cell.
extern "C" int64_t schur_footprint_bytes(int ndim, const int64_t dims[3], int precision) {
    const int64_t nc = dims[0] * dims[1] * (ndim == 3 ? dims[2] : 1);
    const int64_t nf = (int64_t)ndim * ((nc + 63) / 64 * 64);
    int64_t b = nf * (1 + 8 + 4 + 1 + 4 * 8 + 8 * ndim) + nc * (1 + 24 + 4 + 4 + 9 * 8 + 8 * ndim + 4);
    if (precision == SCHUR_MIXED) b += nf * 4 * 4 + nc * 5 * 4;
    return b + (4 << 20);
}

extern "C" int schur_server_create(const schur_opts* opts, int64_t mem_budget_bytes,
                                   int max_active, schur_server_t* out) {
    if (!out || mem_budget_bytes <= 0 || max_active < 1)
        return schur_set_error_internal(SCHUR_EINVAL, "bad server arguments");
    schur_opts o;
    if (opts) o = *opts; else schur_opts_default(&o);
    o.loop_mode = SCHUR_LOOP_GRAPH;
    int rc = check_opts(o);
    if (rc) return rc;
    schur_server* s = new schur_server();
    s->opts = o;
    s->budget = mem_budget_bytes;
    s->max_active = max_active;
    s->t0 = Clock::now();
    *out = s;
    return SCHUR_OK;
}

extern "C" int schur_server_submit(schur_server_t s, const uint8_t* host_mask, int ndim,
                                   const int64_t dims[3], const int periodic[3], int axis,
                                   int64_t* job_id) {
    if (!s || !host_mask || !dims || !periodic) return schur_set_error_internal(SCHUR_EINVAL, "null argument");
    if ((ndim != 2 && ndim != 3) || axis < 0 || axis >= ndim)
        return schur_set_error_internal(SCHUR_EINVAL, "bad ndim or axis");
    Job j;
    j.id = s->next_id++;
    j.ndim = ndim;
    for (int a = 0; a < 3; ++a) {
        j.dims[a] = (a < ndim) ? dims[a] : 1;
        j.periodic[a] = periodic[a];
    }
    for (int a = 0; a < ndim; ++a)
        if (j.dims[a] < 2) return schur_set_error_internal(SCHUR_EINVAL, "every extent must be >= 2");
    const int64_t nc = j.dims[0] * j.dims[1] * j.dims[2];
    j.mask.assign(host_mask, host_mask + nc);
    j.axis = axis;
    j.precond = s->opts.precond;
    if (j.precond == SCHUR_PRECOND_AUTO) {
        const int64_t fluid = std::count(j.mask.begin(), j.mask.end(), (uint8_t)1);
        j.precond = (double)fluid < SCHUR_AUTO_SIMPLE_BELOW * (double)nc ? SCHUR_SIMPLE : SCHUR_UZAWA;
    }
    j.bytes = schur_footprint_bytes(ndim, j.dims, s->opts.precision);
    if (s->opts.inner_precond == SCHUR_INNER_MG) {
        // multigrid hierarchies: per fine entry 16 bytes (weights, work vectors, FP32
        // residual), and coarse levels of at most 1/7 of the fine entries at ~104 bytes
        const int64_t nc = j.dims[0] * j.dims[1] * (ndim == 3 ? j.dims[2] : 1);
        const int64_t nf = (int64_t)ndim * nc;
        j.bytes += 16 * (nf + nc) + 104 * (nf + nc) / 7 + (1 << 20);
    }
    if (j.bytes > s->budget) return schur_set_error_internal(SCHUR_ENOMEM, "job larger than the memory budget");
    j.t_submit = now_s(s);
    if (job_id) *job_id = j.id;
    s->pending.push_back(std::move(j));
    return SCHUR_OK;
}

static void finish_job(schur_server* s, Job& j, int status, const schur_stats* st) {
    schur_job_result r;
    std::memset(&r, 0, sizeof(r));
    r.id = j.id;
    r.status = status;
    r.t_submit = j.t_submit;
    r.t_start = j.t_start;
    r.t_done = now_s(s);
    r.bytes = j.bytes;
    r.precond = j.precond;
    if (j.geom) {
        double k = 0.0;
        if (status == SCHUR_OK || status == SCHUR_ENOTCONV) schur_permeability(j.geom, j.axis, &k);
        r.k = k;
        schur_destroy(j.geom);
        j.geom = nullptr;
    }
    if (st) {
        r.outer_iters = st->outer_iters;
        r.inner_iters = st->inner_iters_A + st->inner_iters_A_f32 + st->inner_iters_S +
                        st->inner_iters_S_f32;
    }
    if (j.stream) cudaStreamDestroy(j.stream);
    j.stream = nullptr;
    s->used -= j.bytes;
    s->done.push_back(r);
}

// Admit what fits, collect what finished.  Never blocks on the GPU.
extern "C" int schur_server_progress(schur_server_t s, int* n_active, int* n_pending) {
    NvtxRange nvtx_("schur_server_progress");
    if (!s) return schur_set_error_internal(SCHUR_EINVAL, "null server");
    // completions
    for (size_t i = 0; i < s->active.size();) {
        Job& j = s->active[i];
        int done = 0;
        int rc = schur_query(j.geom, &done);
        if (rc != SCHUR_OK) done = 1;
        if (!done) { ++i; continue; }
        schur_stats st;
        std::memset(&st, 0, sizeof(st));
        const int status = rc != SCHUR_OK ? rc : schur_finish(j.geom, &st, nullptr);
        finish_job(s, j, status, &st);
        s->active.erase(s->active.begin() + i);
    }
    // admissions, in arrival order
    while (!s->pending.empty() && (int)s->active.size() < s->max_active &&
           s->used + s->pending.front().bytes <= s->budget) {
        Job j = std::move(s->pending.front());
        s->pending.pop_front();
        j.t_start = now_s(s);
        s->used += j.bytes;
        int rc = SCHUR_OK;
        if (cudaStreamCreateWithFlags(&j.stream, cudaStreamNonBlocking) != cudaSuccess)
            rc = schur_set_error_internal(SCHUR_ECUDA, "stream create");
        if (rc == SCHUR_OK)
            rc = schur_create_geometry(j.mask.data(), j.ndim, j.dims, j.periodic, j.stream, &j.geom);
        if (rc == SCHUR_OK)
            rc = set_launch_shape(handle_of(j.geom), s->shape[0], s->shape[1], s->shape[2]);
        if (rc == SCHUR_OK) {
            double f[3] = {0.0, 0.0, 0.0};
            f[j.axis] = 1.0;
            rc = schur_set_force(j.geom, f);
        }
        if (rc == SCHUR_OK) {
            schur_opts o = s->opts;
            o.precond = j.precond;
            rc = schur_solve_async(j.geom, &o);
        }
        j.mask.clear();
        j.mask.shrink_to_fit();
        if (rc != SCHUR_OK) {
            finish_job(s, j, rc, nullptr);
            continue;
        }
        s->active.push_back(std::move(j));
    }
    s->peak_used = std::max(s->peak_used, s->used);
    s->peak_active = std::max(s->peak_active, (int)s->active.size());
    if (n_active) *n_active = (int)s->active.size();
    if (n_pending) *n_pending = (int)s->pending.size();
    return SCHUR_OK;
}

// Move up to max finished results into out; *n_out gets the count.
extern "C" int schur_server_take(schur_server_t s, schur_job_result* out, int max, int* n_out) {
    if (!s || !n_out || (max > 0 && !out)) return schur_set_error_internal(SCHUR_EINVAL, "null argument");
    const int n = std::min<int>(max, (int)s->done.size());
    for (int i = 0; i < n; ++i) out[i] = s->done[i];
    s->done.erase(s->done.begin(), s->done.begin() + n);
    *n_out = n;
    return SCHUR_OK;
}

extern "C" int schur_server_info(schur_server_t s, int64_t* peak_bytes, int* peak_active) {
    if (!s) return schur_set_error_internal(SCHUR_EINVAL, "null server");
    if (peak_bytes) *peak_bytes = s->peak_used;
    if (peak_active) *peak_active = s->peak_active;
    return SCHUR_OK;
}

extern "C" void schur_server_destroy(schur_server_t s) {
    if (!s) return;
    for (Job& j : s->active) {
        if (j.geom) schur_destroy(j.geom);
        if (j.stream) cudaStreamDestroy(j.stream);
    }
    delete s;
}
