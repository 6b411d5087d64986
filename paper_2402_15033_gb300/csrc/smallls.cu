// Small dense steps of the s-step GMRES cycle (one CTA): see smallls_body.cuh.
#include "smallls_body.cuh"

namespace gm {

namespace {

__global__ void cycle_begin_kernel(DevState* st, CycleBasis cb) {
    if (threadIdx.x == 0) {
        st->s = cb.s;
        st->panel = cb.panel;
        st->sigma = cb.sigma;
        st->cheb = cb.cheb;
    }
    if (threadIdx.x < 16) st->theta[threadIdx.x] = cb.theta[threadIdx.x];
    cycle_begin_body(st, 0);
}

__global__ void __launch_bounds__(kLsThreads) hessenberg_ls_kernel(DevState* st, int lo, int t) {
    extern __shared__ __align__(16) double ls_dyn[];
    hessenberg_ls_body(st, lo, t, ls_dyn);
}

__global__ void __launch_bounds__(256) bcgs2_combine_kernel(const DevState* st, int k, int s, const double* S,
                                                            double* R) {
    bcgs2_combine_body(st, k, s, S, R);
}

__global__ void __launch_bounds__(256) eye_panel_kernel(DevState* st, int lo, int t) { eye_panel_body(st, lo, t); }

__global__ void __launch_bounds__(256) pip3_combine_kernel(DevState* st, int lo, int t, const double* Sb,
                                                           const double* Sc, double* Su, double* Sp) {
    pip3_combine_body(st, lo, t, Sb, Sc, Su, Sp);
}

}  // namespace

cudaError_t launch_cycle_begin(cudaStream_t st, DevState* ds, const CycleBasis& cb) {
    cycle_begin_kernel<<<1, 64, 0, st>>>(ds, cb);
    return cudaGetLastError();
}

cudaError_t launch_hessenberg_ls(cudaStream_t st, DevState* ds, int lo, int t) {
    static const cudaError_t attr = smem_limit(hessenberg_ls_kernel, hessenberg_ls_smem());
    if (attr != cudaSuccess) return attr;
    hessenberg_ls_kernel<<<1, kLsThreads, hessenberg_ls_smem(), st>>>(ds, lo, t);
    return cudaGetLastError();
}

cudaError_t launch_bcgs2_combine(cudaStream_t st, const DevState* ds, int k, int s, const double* S, double* R) {
    bcgs2_combine_kernel<<<1, 256, 0, st>>>(ds, k, s, S, R);
    return cudaGetLastError();
}

cudaError_t launch_pip3_combine(cudaStream_t st, DevState* ds, int lo, int t, const double* S) {
    const size_t SB = (size_t)kLsLd * kLsLd;
    pip3_combine_kernel<<<1, 256, 0, st>>>(ds, lo, t, S, S + SB, const_cast<double*>(S) + 2 * SB,
                                           const_cast<double*>(S) + 3 * SB);
    return cudaGetLastError();
}

cudaError_t launch_eye_panel(cudaStream_t st, DevState* ds, int lo, int t) {
    eye_panel_kernel<<<1, 256, 0, st>>>(ds, lo, t);
    return cudaGetLastError();
}

}  // namespace gm
