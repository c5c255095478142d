// Host-side interface between the C ABI (api.cu) and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <utility>
#include <vector>

#include "../../include/schur.h"
#include "common.cuh"

namespace schur {

// NVTX range over one library call (shows the call in nsys/ncu timelines; a no-op when no
// tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Multigrid hierarchy of one inner operator (A or S-hat_simple), built by mg.cu.  Level 0
// is the fine operator in the compact layout; levels 1 .. nlev-1 are Galerkin operators of
// 2 x 2 x 2 aggregates stored as 7-point tables, the last one diagonal.
struct MgOp {
    int nlev = 0;                  // levels including the fine one (0: not built)
    int tail = 0;                  // first level that one block runs alone in the loop kernel
    int ch16 = 0;                  // the first tail level's children fit 16-bit shared-memory slots
    std::vector<long long> n;      // entries per level
    void* lev = nullptr;           // device array of the levels' descriptors (FP32 cycle)
    void* img = nullptr;           // tables of the tail levels in their shared-memory layout
    std::vector<int> off;          // shared-memory slot offset of each tail level
    float* r32 = nullptr;          // [n_0 + 1] FP32 copy of an FP64 inner residual
    std::vector<void*> bufs;       // every device buffer of the hierarchy
    long long bytes = 0;
};

// Device buffers and graphs of one geometry (the object behind schur_geom_t).
struct Handle {
    Dev g{};
    cudaStream_t stream = nullptr;
    int nsm = 152;
    int target_blocks = 1216;    // grid cap: blocks per SM of the launch shape x SMs
    int min_per_thread = 1;      // grids also give every thread at least this many entries
    bool persistent = true;      // inner solves: one cooperative loop kernel (else one graph
                                 // node per phase inside a conditional while node)

    uint8_t* mask = nullptr;     // [ncell]
    uint8_t* flags = nullptr;    // [d][stride]
    double* invdS = nullptr;     // [ncell] inverse diagonal of S-hat_simple (0 off fluid)
    // inner A solve (face space)
    double *ax = nullptr, *ar = nullptr, *ap = nullptr, *aq = nullptr;
    // inner SIMPLE solve (cell space)
    double *sx = nullptr, *sr = nullptr, *sp = nullptr, *sq = nullptr;
    // outer Schur CG (cell space)
    double *op = nullptr, *orr = nullptr, *od = nullptr, *oq = nullptr, *og = nullptr;
    double* u = nullptr;         // recovered velocity [d][stride]
    // FP32 inner solves of the mixed-precision path (allocated on first use)
    float *axf = nullptr, *arf = nullptr, *apf = nullptr, *aqf = nullptr;
    float *sxf = nullptr, *srf = nullptr, *spf = nullptr, *sqf = nullptr, *invdSf = nullptr;
    // connected fluid components (connectivity through unknown faces)
    int* cmpc = nullptr;         // [n_p] component id of each fluid cell (compact order)
    double* cmean = nullptr;     // [n_comp] per-component mean of the last projected vector
    int* small_start = nullptr;  // [n_small + 1] CSR offsets of the small components
    int* small_cells = nullptr;  // compact indices of the small components' cells
    int n_comp = 0, n_big = 0, n_small = 0;
    // compact layout of the inner solves: unknown faces in (a, z, y, x) order and fluid
    // cells in (z, y, x) order; per row of nx positions a bitmap word and the compact
    // index of the word's first set bit, so that a neighbour's compact index is a popcount
    uint32_t* ulist = nullptr;   // [n_u] face index (into [d][stride]) of unknown k
    uint32_t* flist = nullptr;   // [n_p] cell index of fluid cell m
    uint8_t* ufl = nullptr;      // [n_u] flag byte of unknown k
    uint32_t *fmask = nullptr, *fbase = nullptr;  // face rows: [d * nz * ny][W]
    uint32_t *cmask = nullptr, *cbase = nullptr;  // cell rows: [nz * ny][W]
    int W = 1;                   // 32-bit words per row
    // neighbour tables of the stencils, built once per geometry from the bitmaps (row e
    // of a table holds, for every entry, the compact index of its neighbour in direction
    // e = 2 axis + (0: minus, 1: plus); a missing neighbour points at the entry one past
    // the end of the vectors, which is kept at 0)
    uint32_t* nbA = nullptr;     // [2d][ldA] neighbour faces of unknown k
    uint32_t* nbS = nullptr;     // [2d][ldS] neighbour cells of fluid cell m across open faces
    uint32_t* codeS = nullptr;   // [n_p] 3 bits per direction: 0 closed, 1 + ghost count open
    double* dSc = nullptr;       // [n_p] diagonal of S-hat_simple, compact
    long long ldA = 0, ldS = 0;
    double* invdSc = nullptr;    // [n_p] inverse S-hat diagonal, compact
    double* stage = nullptr;     // [d][stride] staging of schur_solve_A's right-hand side
    long long n_u = 0, n_p = 0;
    double* partials = nullptr;  // reduction scratch
    double* hist = nullptr;      // [hist_cap][4] per-iteration record of the outer loop
    int hist_cap = 0;
    Ctl* dctl = nullptr;         // device control block
    Ctl* hctl = nullptr;         // pinned host shadow

    cudaGraph_t graph_solve[4] = {nullptr, nullptr, nullptr, nullptr};      // [precision][precond]
    cudaGraphExec_t exec_solve[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaGraph_t graph_recover = nullptr;
    cudaGraphExec_t exec_recover = nullptr;
    cudaGraph_t graph_solo = nullptr;
    cudaGraphExec_t exec_solo = nullptr;
    cudaGraph_t graph_full[4] = {nullptr, nullptr, nullptr, nullptr};  // solve + recover
    cudaGraphExec_t exec_full[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t done_ev = nullptr;    // end of an asynchronous solve
    bool pending = false;             // an asynchronous solve is in flight
    int pending_precision = 0;
    int next_slot = 0;
    std::vector<std::pair<int, unsigned long long>> handles;

    // multigrid inner preconditioner: hierarchies of A and S-hat (built on first use) and
    // the inner preconditioner of the recorded graphs (SCHUR_INNER_*)
    MgOp mgA, mgS;
    int inner_precond = 0;

    double force[3] = {1.0, 0.0, 0.0};
    bool solved = false, recovered = false;
    int last_loop = 0;
    int last_precision = 0;
    long long bytes = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

// geometry.cu
cudaError_t launch_flags(Handle& H);
cudaError_t launch_invdiag_simple(Handle& H);
cudaError_t launch_apply_A(Handle& H, const double* x, double* y);
cudaError_t launch_apply_B(Handle& H, const double* u, double* p);
cudaError_t launch_apply_BT(Handle& H, const double* p, double* u);
cudaError_t launch_apply_simple(Handle& H, const double* p, double* q);
cudaError_t launch_to_float(Handle& H, const double* src, float* dst, long long n);
cudaError_t launch_gather_u8(Handle& H, const uint8_t* src, const uint32_t* idx, uint8_t* dst, long long n);
cudaError_t launch_gather_f64(Handle& H, const double* src, const uint32_t* idx, double* dst, long long n);
cudaError_t launch_scatter_f64(Handle& H, const double* src, const uint32_t* idx, double* dst, long long n);

// krylov.cu: fill nbA, nbS, codeS and dSc from the row bitmaps and the face flags
cudaError_t launch_build_tables(Handle& H);

// krylov.cu: record the control flow of a call into R (graph nodes or direct launches)
void record_solve(Handle& H, Recorder& R, int precond, int precision);
void record_recover(Handle& H, Recorder& R);
void record_solve_recover(Handle& H, Recorder& R, int precond, int precision);
void record_solve_A(Handle& H, Recorder& R, const double* b, double* x);
cudaError_t time_kernel(Handle& H, int which, int slot, float* ms);
cudaError_t measure_fp64_peak(cudaStream_t s, int iters, double* lane_ops_per_s);

// mg.cu: build the multigrid hierarchy of A (simple = false) or S-hat (simple = true) when
// missing (returns a SCHUR_* code); record the
// persistent multigrid-preconditioned CG loop of one inner solve (after its init kernel);
// free a hierarchy.
int mg_prepare(Handle& H, bool simple);
void record_mg_loop(Handle& H, Recorder& R, bool simple, bool fp32, void* x, void* r, void* p,
                    void* q, CgState* st, const int* gate);
void mg_free(MgOp& M);

}  // namespace schur

// api.cu: record an error for schur_last_error() and return `code`
int schur_set_error_internal(int code, const char* msg);

// api.cu: pieces of a solve shared by the synchronous, asynchronous, batched and served
// paths.
namespace schur {
int check_opts(const schur_opts& o);
// SCHUR_PRECOND_AUTO resolved for this geometry (SIMPLE below the fluid-fraction threshold).
schur_opts resolve_precond(const Handle& H, schur_opts o);
int prepare_solve(Handle& H, const schur_opts& o, int use_graph);
int upload_ctl(Handle& H);
int download_ctl_async(Handle& H);
void fill_solve_stats(Handle& H, int precision, schur_stats* stats);
void fill_recover_stats(Handle& H, schur_stats* stats);
Handle& handle_of(schur_geom_t g);
// Set the launch shape of a handle's kernels and drop its recorded graphs.
int set_launch_shape(Handle& H, int blocks_per_sm, int entries_per_thread, int persistent);
}  // namespace schur
