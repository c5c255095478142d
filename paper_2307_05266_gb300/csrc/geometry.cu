// Face flags (geometry -> MAC unknowns) and the single matrix-free operators
// A, B, B^T and S-hat_simple.
//
// Discretisation (Section 2.1 MAC placement, eq. coupled_matrix, eq. interior_boundary):
//   face (a, c) lies between cells c - e_a and c; it is an unknown when both are fluid.
//   (A u)_f = h^-2 ((2d + g_f) u_f - sum of the unknown neighbour faces of the same
//   component), where g_f counts the tangential neighbour faces with two solid cells
//   (ghost value -u_f behind a wall half a cell away); neighbours that are wall faces
//   hold u = 0.  (B u)_c = -h^-1 sum_a (u_(a,c+e_a) - u_(a,c));
//   (B^T p)_(a,c) = h^-1 (p_c - p_(c-e_a)).
//   S-hat_simple = B diag(A)^-1 B^T (eq. schur_uzawa_prec):
//   (S-hat p)_c = sum over the unknown faces f of c of (p_c - p_nb(f)) / (2d + g_f).
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

static inline dim3 tile_block() { return dim3(kTileX, kTileY, 1); }
static inline unsigned tile_grid(const Handle& H) {
    const long long gx = (H.g.nx + kTileX - 1) / kTileX, gy = (H.g.ny + kTileY - 1) / kTileY;
    long long nt = gx * gy * H.g.nz;
    return (unsigned)(nt < H.target_blocks ? nt : H.target_blocks);
}

__device__ __forceinline__ int fluid_at(const Dev& g, const uint8_t* m, int x, int y, int z) {
    long long c = cell_at(g, x, y, z);
    return c < 0 ? 0 : (m[c] == 1);
}

// One thread per cell: flags of the d faces (a, c), plus counts of unknown faces per axis,
// fluid cells and mask bytes other than 0/1.
__global__ void k_flags(Dev g, const uint8_t* __restrict__ mask, uint8_t* __restrict__ flags,
                        Ctl* ctl, double* partials) {
    count_launch(ctl);
    double v[5] = {0, 0, 0, 0, 0};
    TILE_LOOP_BEGIN(g)
        const uint8_t mc = mask[c];
        if (mc > 1) v[4] += 1.0;
        const int fc = (mc == 1);
        v[3] += fc;
        for (int a = 0; a < g.d; ++a) {
            int ex, ey, ez;
            axis_step(a, 1, ex, ey, ez);
            const int lower = fluid_at(g, mask, x - ex, y - ey, z - ez);
            uint8_t f = 0;
            if (fc && lower) {
                int ghosts = 0;
                for (int b = 0; b < g.d; ++b) {
                    if (b == a) continue;
                    for (int s = -1; s <= 1; s += 2) {
                        int bx, by, bz;
                        axis_step(b, s, bx, by, bz);
                        const int up = fluid_at(g, mask, x + bx, y + by, z + bz);
                        const int lo = fluid_at(g, mask, x + bx - ex, y + by - ey, z + bz - ez);
                        ghosts += (!up && !lo);
                    }
                }
                f = (uint8_t)(1 | (ghosts << 1));
                v[a] += 1.0;
            }
            flags[(long long)a * g.stride + c] = f;
        }
    TILE_LOOP_END
    if (reduce_last_block<5>(v, partials, &ctl->ticket)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            for (int k = 0; k < 5; ++k) ctl->counts[k] = v[k];
            ctl->n_fluid = v[3];
        }
    }
}

__device__ __forceinline__ double face_val(const Dev& g, const uint8_t* __restrict__ flags,
                                           const double* __restrict__ u, int a, int x, int y,
                                           int z) {
    long long c = cell_at(g, x, y, z);
    if (c < 0) return 0.0;
    const long long i = (long long)a * g.stride + c;
    return (flags[i] & 1) ? u[i] : 0.0;
}

__device__ __forceinline__ double face_inv_diag(const Dev& g, uint8_t f) {
    return 1.0 / (double)(2 * g.d + (f >> 1));
}

__global__ void k_invdiag_simple(Dev g, const uint8_t* __restrict__ mask,
                                 const uint8_t* __restrict__ flags, double* __restrict__ invd,
                                 Ctl* ctl) {
    count_launch(ctl);
    TILE_LOOP_BEGIN(g)
        double s = 0.0;
        if (mask[c] == 1) {
            for (int a = 0; a < g.d; ++a) {
                int ex, ey, ez;
                axis_step(a, 1, ex, ey, ez);
                const uint8_t fl = flags[(long long)a * g.stride + c];
                if (fl & 1) s += face_inv_diag(g, fl);
                const long long cu = cell_at(g, x + ex, y + ey, z + ez);
                if (cu >= 0) {
                    const uint8_t fu = flags[(long long)a * g.stride + cu];
                    if (fu & 1) s += face_inv_diag(g, fu);
                }
            }
        }
        invd[c] = s > 0.0 ? 1.0 / s : 0.0;
    TILE_LOOP_END
}

__global__ void k_apply_A(Dev g, const uint8_t* __restrict__ flags, const double* __restrict__ xin,
                          double* __restrict__ yout, Ctl* ctl) {
    count_launch(ctl);
    TILE_LOOP_BEGIN(g)
        for (int a = 0; a < g.d; ++a) {
            const long long i = (long long)a * g.stride + c;
            const uint8_t f = flags[i];
            double out = 0.0;
            if (f & 1) {
                double s = face_val(g, flags, xin, a, x - 1, y, z) + face_val(g, flags, xin, a, x + 1, y, z);
                s += face_val(g, flags, xin, a, x, y - 1, z) + face_val(g, flags, xin, a, x, y + 1, z);
                if (g.d == 3)
                    s += face_val(g, flags, xin, a, x, y, z - 1) + face_val(g, flags, xin, a, x, y, z + 1);
                out = g.h2inv * ((double)(2 * g.d + (f >> 1)) * xin[i] - s);
            }
            yout[i] = out;
        }
    TILE_LOOP_END
}

__global__ void k_apply_B(Dev g, const uint8_t* __restrict__ mask, const uint8_t* __restrict__ flags,
                          const double* __restrict__ u, double* __restrict__ p, Ctl* ctl) {
    count_launch(ctl);
    TILE_LOOP_BEGIN(g)
        double out = 0.0;
        if (mask[c] == 1) {
            double s = 0.0;
            for (int a = 0; a < g.d; ++a) {
                int ex, ey, ez;
                axis_step(a, 1, ex, ey, ez);
                s += face_val(g, flags, u, a, x + ex, y + ey, z + ez) - face_val(g, flags, u, a, x, y, z);
            }
            out = -g.hinv * s;
        }
        p[c] = out;
    TILE_LOOP_END
}

__global__ void k_apply_BT(Dev g, const uint8_t* __restrict__ flags, const double* __restrict__ p,
                           double* __restrict__ u, Ctl* ctl) {
    count_launch(ctl);
    TILE_LOOP_BEGIN(g)
        for (int a = 0; a < g.d; ++a) {
            const long long i = (long long)a * g.stride + c;
            double out = 0.0;
            if (flags[i] & 1) {
                int ex, ey, ez;
                axis_step(a, 1, ex, ey, ez);
                out = g.hinv * (p[c] - p[cell_at(g, x - ex, y - ey, z - ez)]);
            }
            u[i] = out;
        }
    TILE_LOOP_END
}

__global__ void k_apply_simple(Dev g, const uint8_t* __restrict__ mask,
                               const uint8_t* __restrict__ flags, const double* __restrict__ p,
                               double* __restrict__ q, Ctl* ctl) {
    count_launch(ctl);
    TILE_LOOP_BEGIN(g)
        double out = 0.0;
        if (mask[c] == 1) {
            const double pc = p[c];
            for (int a = 0; a < g.d; ++a) {
                int ex, ey, ez;
                axis_step(a, 1, ex, ey, ez);
                const uint8_t fl = flags[(long long)a * g.stride + c];
                if (fl & 1) out += (pc - p[cell_at(g, x - ex, y - ey, z - ez)]) * face_inv_diag(g, fl);
                const long long cu = cell_at(g, x + ex, y + ey, z + ez);
                if (cu >= 0) {
                    const uint8_t fu = flags[(long long)a * g.stride + cu];
                    if (fu & 1) out += (pc - p[cu]) * face_inv_diag(g, fu);
                }
            }
        }
        q[c] = out;
    TILE_LOOP_END
}

__global__ void k_to_float(const double* __restrict__ src, float* __restrict__ dst, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

__global__ void k_gather_u8(const uint8_t* __restrict__ src, const uint32_t* __restrict__ idx,
                            uint8_t* __restrict__ dst, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = src[idx[i]];
}
__global__ void k_gather_f64(const double* __restrict__ src, const uint32_t* __restrict__ idx,
                             double* __restrict__ dst, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = src[idx[i]];
}
__global__ void k_scatter_f64(const double* __restrict__ src, const uint32_t* __restrict__ idx,
                              double* __restrict__ dst, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[idx[i]] = src[i];
}
cudaError_t launch_gather_u8(Handle& H, const uint8_t* src, const uint32_t* idx, uint8_t* dst, long long n) {
    k_gather_u8<<<H.target_blocks, kBlock, 0, H.stream>>>(src, idx, dst, n);
    return cudaGetLastError();
}
cudaError_t launch_gather_f64(Handle& H, const double* src, const uint32_t* idx, double* dst, long long n) {
    k_gather_f64<<<H.target_blocks, kBlock, 0, H.stream>>>(src, idx, dst, n);
    return cudaGetLastError();
}
cudaError_t launch_scatter_f64(Handle& H, const double* src, const uint32_t* idx, double* dst, long long n) {
    k_scatter_f64<<<H.target_blocks, kBlock, 0, H.stream>>>(src, idx, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_to_float(Handle& H, const double* src, float* dst, long long n) {
    k_to_float<<<H.target_blocks, kBlock, 0, H.stream>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_flags(Handle& H) {
    k_flags<<<tile_grid(H), tile_block(), 0, H.stream>>>(H.g, H.mask, H.flags, H.dctl, H.partials);
    return cudaGetLastError();
}
cudaError_t launch_invdiag_simple(Handle& H) {
    k_invdiag_simple<<<tile_grid(H), tile_block(), 0, H.stream>>>(H.g, H.mask, H.flags, H.invdS, H.dctl);
    return cudaGetLastError();
}
cudaError_t launch_apply_A(Handle& H, const double* x, double* y) {
    k_apply_A<<<tile_grid(H), tile_block(), 0, H.stream>>>(H.g, H.flags, x, y, H.dctl);
    return cudaGetLastError();
}
cudaError_t launch_apply_B(Handle& H, const double* u, double* p) {
    k_apply_B<<<tile_grid(H), tile_block(), 0, H.stream>>>(H.g, H.mask, H.flags, u, p, H.dctl);
    return cudaGetLastError();
}
cudaError_t launch_apply_BT(Handle& H, const double* p, double* u) {
    k_apply_BT<<<tile_grid(H), tile_block(), 0, H.stream>>>(H.g, H.flags, p, u, H.dctl);
    return cudaGetLastError();
}
cudaError_t launch_apply_simple(Handle& H, const double* p, double* q) {
    k_apply_simple<<<tile_grid(H), tile_block(), 0, H.stream>>>(H.g, H.mask, H.flags, p, q, H.dctl);
    return cudaGetLastError();
}

}  // namespace schur
