// sw_internal.h -- host-side interfaces between the C ABI (sw_api.cu) and the
// kernel translation units (sw_solver.cu, sw_setup.cu, sw_static.cu).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace sw {

struct EnsDesc;

template <class CT>
struct OpArgs {
    int nx, ny;
    const CT *ax, *cx, *bx, *ay, *cy, *by, *C;
};

struct FaceArgs {
    int nx, ny;
    double dlam, dphi;
    const double *A11, *A12, *A21, *A22, *B1, *B2, *C;       // caller, cell-centred
    double *ax, *cx, *bx, *ay, *cy, *by, *C64, *diag;        // FP64 faces, diag(L)
    float *wax, *wcx, *wbx, *way, *wcy, *wby, *wC, *wdiag;   // FP32 copies
    double *rowmax;                                          // max |diag(P^M)| per row
};

struct FactorArgs {
    int nx, ny;
    double eta_explicit;            // > 0: use it; otherwise 1/max|diag(P^M)|
    const double *ax, *C, *rowmax;
    double *lf, *invD, *zz, *gam, *ec, *eta_out;
    float *lf32, *invD32, *zz32;
};

cudaError_t launch_faces(const FaceArgs &a, int threads, cudaStream_t s);
cudaError_t launch_factor(const FactorArgs &a, int threads, cudaStream_t s);
size_t gcr_smem_bytes(int prec, int max_nx, int k, int cache_const, int cache_state);
cudaError_t gcr_occupancy(int prec, int k, int threads, size_t smem, int *blocks_per_sm);
cudaError_t launch_gcr(int prec, int k, const EnsDesc *Ddev, int grid, int max_nx, int threads, size_t smem,
                       cudaStream_t s);
cudaError_t launch_operator_f64(const OpArgs<double> &a, const double *x, double *y, int threads, cudaStream_t s);
cudaError_t launch_operator_f32(const OpArgs<float> &a, const float *x, float *y, int threads, cudaStream_t s);
cudaError_t launch_precond(int prec, const void *Mdev, int nx, int ny, int nstages, void *qout, int threads,
                           cudaStream_t s);
cudaError_t launch_fill(double *p, size_t n, double v, cudaStream_t s);
size_t member_dev_bytes(int prec);
// the fixed scratch of sw_gcr_solve_noalloc on the current device (sw_static.cu)
cudaError_t noalloc_scratch(void **ptr, size_t *bytes);

} // namespace sw
