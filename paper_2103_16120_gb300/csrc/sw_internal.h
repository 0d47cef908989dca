// sw_internal.h -- host-side interfaces between the C ABI (sw_api.cu) and the
// kernel translation units (sw_solver.cu, sw_setup.cu, sw_static.cu).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "../../include/sw_elliptic.h"

struct sw_grid_s;
struct sw_model_s;

namespace sw {

struct EnsDesc;
struct InitOneArgs;

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
    double *lf, *invD, *zz, *gam, *ec, *eta_out;        // FP64 factors
    float *lf32, *invD32, *zz32;                         // FP32 factors
    double *gam32, *ec32;                                // per row, of the FP32 factors
    // the factors transposed per row for the warp-per-row solver (or null):
    // point i at (i % m) * 32 + i / m, m = nx / 32
    double *lfT, *invDT, *zzT;
    float *lf32T, *invD32T, *zz32T;
};

// geometry of a grid handle, for translation units outside sw_api.cu
struct GridGeom {
    int nx, ny, sms;
    double radius;
};
GridGeom grid_geom(const ::sw_grid_s *g);

// split fluid thickness of Sec. 4.2, Eq. 14 (sw_solver.cu)
struct SplitRefreshArgs {
    int nx, ny;
    const double *phi;
    float *hat, *dx, *cx, *dy, *cy;
};
struct SplitResidualArgs {
    int nx, ny;
    const double *phi, *R;
    float *r;
    const float *wax, *wcx, *wbx, *way, *wcy, *wby, *wC;
    const float *hat, *dx, *cx, *dy, *cy;
};
cudaError_t launch_split_refresh(const SplitRefreshArgs &a, cudaStream_t s);
cudaError_t launch_split_residual(const SplitResidualArgs &a, cudaStream_t s);

cudaError_t launch_faces(const FaceArgs &a, int threads, cudaStream_t s);
cudaError_t launch_factor(const FactorArgs &a, bool fp64, int threads, cudaStream_t s);
size_t gcr_smem_bytes(int prec, int max_nx, int k, int cache_const, int cache_state);
// shared memory of the warp-per-row mode (0 when nx does not allow it)
size_t gcr_warp_smem_bytes(int prec, int nx, int threads, int stage);
cudaError_t gcr_occupancy(int prec, int k, int minb, int warp, int threads, size_t smem, int *blocks_per_sm);
// Raise kernel f's dynamic shared-memory limit on the current device to at
// least smem bytes.  The limit only grows: a launch recorded in a CUDA graph
// (the ensemble and learned-preconditioner graphs) keeps its size, so a later
// launch must not lower the limit below it.
cudaError_t raise_smem_limit(const void *f, size_t smem);
cudaError_t launch_gcr(int prec, int k, int minb, int warp, const EnsDesc *Ddev, int grid, int max_nx, int threads,
                       size_t smem, cudaStream_t s);
// the instantiations of the GCR kernel, one translation unit each
// (sw_gcr_*.cu): the kernel for a k and register budget, and the unit's
// barrier test hook and time line
#define SW_GCR_UNIT_DECL(TAG)                                                              \
    const void *gcr_kernel_##TAG(int k, int minb);                                         \
    cudaError_t gcr_debug_##TAG(unsigned long long extra, unsigned long long limit_ns);    \
    void gcr_trace_##TAG(unsigned long long *buf, int cap, int block);
SW_GCR_UNIT_DECL(f64)
SW_GCR_UNIT_DECL(f16)
SW_GCR_UNIT_DECL(bf16)
SW_GCR_UNIT_DECL(w64)
SW_GCR_UNIT_DECL(w16)
SW_GCR_UNIT_DECL(wbf16)
SW_GCR_UNIT_DECL(solver)
// the warp-per-row kernels specialised for rows of 32 m points (m = 32, 64;
// GCR k <= 4, one block per SM; null for other m)
const void *gcr_kernel_s16(int m);
const void *gcr_kernel_sbf16(int m);
cudaError_t gcr_debug_s16(unsigned long long extra, unsigned long long limit_ns);
cudaError_t gcr_debug_sbf16(unsigned long long extra, unsigned long long limit_ns);
void gcr_trace_s16(unsigned long long *buf, int cap, int block);
void gcr_trace_sbf16(unsigned long long *buf, int cap, int block);
cudaError_t launch_operator_f64(const OpArgs<double> &a, const double *x, double *y, int threads, cudaStream_t s);
cudaError_t launch_operator_f32(const OpArgs<float> &a, const float *x, float *y, int threads, cudaStream_t s);
cudaError_t launch_precond(int prec, const void *Mdev, int nx, int ny, int nstages, void *qout, int threads,
                           cudaStream_t s);
cudaError_t launch_fill(double *p, size_t n, double v, cudaStream_t s);
cudaError_t set_barrier_debug(unsigned long long extra, unsigned long long limit_ns);
// every member of a launch descriptor: initial GCR state, cleared barrier
cudaError_t launch_init_members(const EnsDesc *Ddev, int n, cudaStream_t s);
// one member: writes its descriptor, the launch descriptor and the initial state
cudaError_t launch_init_one(const InitOneArgs &a, cudaStream_t s);
// the member's e from an FP32 field (the network's direction)
cudaError_t launch_store_e(int prec, const void *Mdev, const float *ef, int nx, int ny, int threads, cudaStream_t s);
// the learned preconditioner applied to the residual r (FP64 or FP32) of
// grid g, e (FP32 [ny][nx]) into the model's buffer, whose address is returned
sw_status model_precondition(::sw_model_s *m, const ::sw_grid_s *g, const void *r, bool r64, float *e,
                             cudaStream_t s);
sw_status model_check_grid(const ::sw_grid_s *g);
float *model_scratch(::sw_model_s *m, int ny, int nx);
// a number that identifies the model and its current activation storage
// (new for every model and at every reallocation of its activations)
unsigned long long model_gen(::sw_model_s *m);
size_t member_dev_bytes(int prec);
// set the calling thread's error message and return st (sw_api.cu)
sw_status api_fail(sw_status st, const char *msg);

// what the learned preconditioner reads from a grid handle (sw_api.cu)
struct GridView {
    int nx, ny, device, sms;
    const float *wax, *way, *wdiag;   // FP32 zonal / meridional face coefficients, diag(L)
};
GridView grid_view(const ::sw_grid_s *g);

// the fixed scratch of sw_gcr_solve_noalloc on the current device (sw_static.cu)
cudaError_t noalloc_scratch(void **ptr, size_t *bytes);

} // namespace sw
