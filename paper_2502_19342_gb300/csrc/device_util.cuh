// Device helpers shared by the forward and adjoint kernels.
#pragma once

#include "common.cuh"

namespace dgfv {

__device__ __forceinline__ const double* B(const Params& P, int32_t off) { return P.bank + off; }

// 2D tensor-product map of a face field in shared memory:
//   out[x][ao + no*bo] = sum_{ai,bi} M[ao][ai] M[bo][bi] in[x][ai + ni*bi],  x < nvar,
// M is no x ni (row-major); tmp holds nvar*no*ni doubles.  All threads of the
// block take part; the call ends with a barrier.
__device__ __forceinline__ void face_map(const double* in, int ni, double* out, int no, const double* M, int nvar,
                                         double* tmp) {
    const int n1 = no * ni;
    for (int i = threadIdx.x; i < nvar * n1; i += blockDim.x) {
        const int x = i / n1, r = i % n1, ao = r % no, bi = r / no;
        const double* src = in + x * ni * ni + ni * bi;
        double s = 0.0;
        for (int ai = 0; ai < ni; ++ai) s = fma(__ldg(M + ao * ni + ai), src[ai], s);
        tmp[x * n1 + ao + no * bi] = s;
    }
    __syncthreads();
    const int n2 = no * no;
    for (int i = threadIdx.x; i < nvar * n2; i += blockDim.x) {
        const int x = i / n2, r = i % n2, ao = r % no, bo = r / no;
        const double* src = tmp + x * n1 + ao;
        double s = 0.0;
        for (int bi = 0; bi < ni; ++bi) s = fma(__ldg(M + bo * ni + bi), src[no * bi], s);
        out[x * n2 + r] = s;
    }
    __syncthreads();
}

// face_map with its own matrix per face direction: Ma (no x ni) along a, Mb
// along b.
__device__ __forceinline__ void face_map2(const double* in, int ni, double* out, int no, const double* Ma,
                                          const double* Mb, int nvar, double* tmp) {
    const int n1 = no * ni;
    for (int i = threadIdx.x; i < nvar * n1; i += blockDim.x) {
        const int x = i / n1, r = i % n1, ao = r % no, bi = r / no;
        const double* src = in + x * ni * ni + ni * bi;
        double s = 0.0;
        for (int ai = 0; ai < ni; ++ai) s = fma(__ldg(Ma + ao * ni + ai), src[ai], s);
        tmp[x * n1 + ao + no * bi] = s;
    }
    __syncthreads();
    const int n2 = no * no;
    for (int i = threadIdx.x; i < nvar * n2; i += blockDim.x) {
        const int x = i / n2, r = i % n2, ao = r % no, bo = r / no;
        const double* src = tmp + x * n1 + ao;
        double s = 0.0;
        for (int bi = 0; bi < ni; ++bi) s = fma(__ldg(Mb + bo * ni + bi), src[no * bi], s);
        out[x * n2 + r] = s;
    }
    __syncthreads();
}

// Transpose of face_map with the same M (no x ni): maps a face field of no^2
// points back to ni^2 points, out = (M^T x M^T) in.
__device__ __forceinline__ void face_map_t(const double* in, int no, double* out, int ni, const double* M, int nvar,
                                           double* tmp) {
    const int n1 = ni * no;
    for (int i = threadIdx.x; i < nvar * n1; i += blockDim.x) {
        const int x = i / n1, r = i % n1, ai = r % ni, bo = r / ni;
        const double* src = in + x * no * no + no * bo;
        double s = 0.0;
        for (int ao = 0; ao < no; ++ao) s = fma(__ldg(M + ao * ni + ai), src[ao], s);
        tmp[x * n1 + ai + ni * bo] = s;
    }
    __syncthreads();
    const int n2 = ni * ni;
    for (int i = threadIdx.x; i < nvar * n2; i += blockDim.x) {
        const int x = i / n2, r = i % n2, ai = r % ni, bi = r / ni;
        const double* src = tmp + x * n1 + ai;
        double s = 0.0;
        for (int bo = 0; bo < no; ++bo) s = fma(__ldg(M + bo * ni + bi), src[ni * bo], s);
        out[x * n2 + r] = s;
    }
    __syncthreads();
}

// Transpose of face_map2 with the same Ma, Mb (no x ni): out = (Ma^T x Mb^T) in.
__device__ __forceinline__ void face_map2_t(const double* in, int no, double* out, int ni, const double* Ma,
                                            const double* Mb, int nvar, double* tmp) {
    const int n1 = ni * no;
    for (int i = threadIdx.x; i < nvar * n1; i += blockDim.x) {
        const int x = i / n1, r = i % n1, ai = r % ni, bo = r / ni;
        const double* src = in + x * no * no + no * bo;
        double s = 0.0;
        for (int ao = 0; ao < no; ++ao) s = fma(__ldg(Ma + ao * ni + ai), src[ao], s);
        tmp[x * n1 + ai + ni * bo] = s;
    }
    __syncthreads();
    const int n2 = ni * ni;
    for (int i = threadIdx.x; i < nvar * n2; i += blockDim.x) {
        const int x = i / n2, r = i % n2, ai = r % ni, bi = r / ni;
        const double* src = tmp + x * n1 + ai;
        double s = 0.0;
        for (int bo = 0; bo < no; ++bo) s = fma(__ldg(Mb + bo * ni + bi), src[ni * bo], s);
        out[x * n2 + r] = s;
    }
    __syncthreads();
}

}  // namespace dgfv
