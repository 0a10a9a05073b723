// adj.cuh -- adjoint-step kernel parameters and host launchers.
#pragma once

#include "swadj_internal.cuh"

namespace swadj {

template <typename R>
struct AdjParams {
    int nx, ny, two_d, order;
    BcSpec bc;
    R nux, nuy;          // dt/dx, dt/dy (fixed step)
    R g, dry_tol;
    const R *src[3];     // (eta~, mu~, gamma~) at step s
    R *dst[3];           // at step s+1
    const R *c;          // double: hbar; float: sqrt(g hbar), 0 where dry
    // fused snapshot (optional): written with the new state when snap_f or
    // snap_d is non-null
    float *snap_f;
    double *snap_d;
    size_t snap_comp_stride;  // elements between components of one snapshot
    double *tau_dev;
    double tau_val;
    // FP32 2D only: take two steps in this launch (the snapshot, if any, is
    // of the state after both)
    int two_steps;
    // FP32 2D one-step kernel: no cell is dry (no wall edges to check)
    int all_wet;
    // FP32 2D one-step kernel: 1 = the unit has had a nonzero value at an
    // earlier step (it skips the quiet scan); null: no quiet scan
    unsigned char *umap;
    int umap_n;
};

template <typename R>
int adj_launch_step(const AdjParams<R> &p, cudaStream_t st);
// entries of the FP32 2D adjoint's unit map
int adj_f32_unit_map_bytes(int nx, int ny);
template <> int adj_launch_step<double>(const AdjParams<double> &, cudaStream_t);
template <> int adj_launch_step<float>(const AdjParams<float> &, cudaStream_t);

// c = sqrt(g hbar) (0 where hbar <= dry_tol), hbar = max(-B, 0) computed from
// the FP64 bathymetry in `B`; atomically maxes c/dx [+ c/dy] into *smax.
template <typename R>
int adj_launch_init(const double *B, R *c, size_t n, int two_d, double g,
                    double dx, double dy, double dry_tol, double *smax,
                    cudaStream_t st);

// Copy the state into snapshot slot `k` (converted to the snapshot type).
template <typename R>
int adj_launch_store(const R *const src[3], int ncomp, size_t n, float *snap_f,
                     double *snap_d, size_t comp_stride, double *tau_dev,
                     double tau_val, cudaStream_t st);

}  // namespace swadj
