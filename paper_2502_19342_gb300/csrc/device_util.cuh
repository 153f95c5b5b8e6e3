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

// The layer of sub-cell means that an FV neighbour sees across face fq of element
// q, on N_FV x N_FV points: an FV element's boundary sub-cell means (its face
// values), or a DG element's solution mapped by V^{DG->FV} (boundary row along
// the face normal, then both face directions).  All threads of the block take
// part; ends with a barrier.
template <int NK>
__device__ __forceinline__ void fv_layer(const Params& P, const double* __restrict__ U, int q, int fq, int n,
                                         double* dst, double* sT1, double* sT2) {
    constexpr int V = NK + 4;
    const int n2 = n * n, d = fq >> 1;
    const int nq = P.t.n[q], nq2 = nq * nq, nq3 = nq2 * nq;
    if (P.t.fv[q]) {
        const double* src = P.b.fu + (P.t.fo[q] + (int64_t)fq * nq2) * V;
        if (nq == n) {
            for (int i = threadIdx.x; i < V * n2; i += blockDim.x) dst[i] = src[i];
            __syncthreads();
        } else {  // per-element counts: the neighbour's layer by its sub-cell overlaps
            for (int i = threadIdx.x; i < V * nq2; i += blockDim.x) sT1[i] = src[i];
            __syncthreads();
            face_map(sT1, nq, dst, n, B(P, P.bi.ov[nq][n]), V, sT2);
        }
        return;
    }
    const double* A = B(P, P.bi.d2f[nq][n]);  // n x nq
    const int row = (fq & 1) ? n - 1 : 0;   // sub-cell layer next to the shared face
    const double* src = U + P.t.off[q];
    for (int i = threadIdx.x; i < V * nq2; i += blockDim.x) {
        const int v = i / nq2, p = i % nq2, a = p % nq, b = p / nq;
        double s = 0.0;
        for (int m = 0; m < nq; ++m)
            s = fma(__ldg(A + row * nq + m), src[(int64_t)v * nq3 + node_index(nq, d, m, a, b)], s);
        sT1[i] = s;
    }
    __syncthreads();
    face_map(sT1, nq, dst, n, A, V, sT2);
}

// The six neighbour layers of FV element e (n sub-cells per direction) into
// sNb (6 x V n^2 conservative values, face-major), with the per-face
// geometry: sID[f] = 1/distance and sGS[f] = rh_d/(l + distance), the
// distance between the boundary sub-cell's centre and the neighbour layer's,
// in e's reference coordinates (l = 2/n).  All six faces at once in three
// passes separated by block barriers:
//   (1) an FV neighbour of the same count: its boundary sub-cell means
//       (its face values) straight into sNb; of another count (per-element
//       counts): its layer into the scratch, mapped by its sub-cell overlaps;
//       a DG neighbour: the boundary row of V^{DG->FV} along the face normal
//       into the scratch, then V^{DG->FV} in both face directions; across a
//       mortar: the values gathered beforehand into the slot;
//   (2), (3) the two face directions of those maps (as face_map).
// sT: 6 V (MAXP^2 + n MAXP) doubles of scratch; sMap, sNq: 6 entries of
// shared memory each.  All threads of the block take part; ends with a
// barrier.
template <int NK>
__device__ __forceinline__ void fv_gather_neighbours(const Params& P, const double* __restrict__ U, int e, int n,
                                                     double* sNb, double* sT, double* sID, double* sGS,
                                                     const double** sMap, int* sNq) {
    constexpr int V = NK + 4;
    const int n2 = n * n;
    const double l = 2.0 / n;
    const double* rh = P.t.rh + 3 * e;
    if (threadIdx.x < 6) {
        const int f = threadIdx.x, q = P.t.nb[6 * e + f];
        int qe = q, nq = n;
        const double* M = nullptr;
        if (q < 0) {
            qe = P.t.mnbe[-1 - q];
        } else if (P.t.fv[q]) {
            nq = P.t.n[q];
            if (nq != n) M = B(P, P.bi.ov[nq][n]);
        } else {
            nq = P.t.n[q];
            M = B(P, P.bi.d2f[nq][n]);
        }
        sMap[f] = M;
        sNq[f] = nq;
        // l/2 (1 + h_neighbour/h), l when the sizes agree; to an FV neighbour
        // with another sub-cell count n_q (per-element counts) l/2 + (h_neighbour/h)/n_q
        const int d = f >> 1;
        const double hr = rh[d] / P.t.rh[3 * qe + d];
        const int nqd = q >= 0 && P.t.fv[q] ? nq : n;
        const double dist = nqd == n ? 0.5 * l * (1.0 + hr) : 0.5 * l + hr / nqd;
        sID[f] = 1.0 / dist;
        sGS[f] = rh[d] / (l + dist);
    }
    __syncthreads();
    const int per_face = V * (MAXP * MAXP + n * MAXP);
    for (int f = 0; f < 6; ++f) {
        const int q = P.t.nb[6 * e + f], fq = f ^ 1, d = f >> 1, nq = sNq[f], nq2 = nq * nq;
        double* dst = sNb + f * V * n2;
        double* lay = sT + f * per_face;
        if (q < 0) {
            const double* src = P.t.mnb + (int64_t)(-1 - q) * V * n2;
            for (int i = threadIdx.x; i < V * n2; i += blockDim.x) dst[i] = src[i];
        } else if (P.t.fv[q]) {
            const double* src = P.b.fu + (P.t.fo[q] + (int64_t)fq * nq2) * V;
            double* to = sMap[f] ? lay : dst;
            for (int i = threadIdx.x; i < V * nq2; i += blockDim.x) to[i] = src[i];
        } else {
            const int nq3 = nq2 * nq, row = (fq & 1) ? n - 1 : 0;  // sub-cell layer next to the shared face
            const double* A = sMap[f];                                // n x nq
            const double* src = U + P.t.off[q];
            for (int i = threadIdx.x; i < V * nq2; i += blockDim.x) {
                const int v = i / nq2, p = i % nq2, a = p % nq, b = p / nq;
                double s = 0.0;
                for (int m = 0; m < nq; ++m)
                    s = fma(__ldg(A + row * nq + m), src[(int64_t)v * nq3 + node_index(nq, d, m, a, b)], s);
                lay[i] = s;
            }
        }
    }
    __syncthreads();
    for (int f = 0; f < 6; ++f) {  // first face direction of the maps: n x nq per variable
        const double* M = sMap[f];
        if (!M) continue;
        const int nq = sNq[f], n1 = n * nq;
        const double* lay = sT + f * per_face;
        double* half = sT + f * per_face + V * MAXP * MAXP;
        for (int i = threadIdx.x; i < V * n1; i += blockDim.x) {
            const int x = i / n1, r = i % n1, ao = r % n, bi = r / n;
            const double* in = lay + x * nq * nq + nq * bi;
            double s = 0.0;
            for (int ai = 0; ai < nq; ++ai) s = fma(__ldg(M + ao * nq + ai), in[ai], s);
            half[x * n1 + ao + n * bi] = s;
        }
    }
    __syncthreads();
    for (int f = 0; f < 6; ++f) {  // second face direction, into the neighbour values
        const double* M = sMap[f];
        if (!M) continue;
        const int nq = sNq[f], n1 = n * nq;
        const double* half = sT + f * per_face + V * MAXP * MAXP;
        double* dst = sNb + f * V * n2;
        for (int i = threadIdx.x; i < V * n2; i += blockDim.x) {
            const int x = i / n2, r = i % n2, ao = r % n, bo = r / n;
            const double* in = half + x * n1 + ao;
            double s = 0.0;
            for (int bi = 0; bi < nq; ++bi) s = fma(__ldg(M + bo * nq + bi), in[n * bi], s);
            dst[x * n2 + r] = s;
        }
    }
    __syncthreads();
}

// Transpose of the neighbour layer an FV element of n sub-cells per direction
// reads across face fq of element q: Ub (the state adjoint of q) += layer^T
// lb, lb the adjoint of the n x n layer.  FV element: its boundary sub-cells
// (with another sub-cell count, per-element counts, the transpose of the
// overlap map first); DG element: V^{DG->FV} transposed in both face
// directions, then the boundary row along the normal.  Ends with a barrier.
template <int NK, bool ATOMIC = false>
__device__ __forceinline__ void fv_layer_t(const Params& P, int q, int fq, int n, const double* lb, double* Ub,
                                           double* sT1, double* sT2) {
    constexpr int V = NK + 4;
    const int d = fq >> 1;
    if (P.t.fv[q]) {
        const int nq = P.t.n[q], nq2 = nq * nq, nq3 = nq2 * nq, m = (fq & 1) ? nq - 1 : 0;
        const double* src = lb;
        if (nq != n) {  // the layer was mapped from q's grid by its overlaps (n x nq)
            face_map_t(lb, n, sT1, nq, B(P, P.bi.ov[nq][n]), V, sT2);
            src = sT1;
        }
        double* dst = Ub + P.t.off[q];
        for (int i = threadIdx.x; i < V * nq2; i += blockDim.x) {
            const int v = i / nq2, p = i % nq2;
            double* t = dst + (int64_t)v * nq3 + node_index(nq, d, m, p % nq, p / nq);
            if (ATOMIC) atomicAdd(t, src[i]);
            else *t += src[i];
        }
        __syncthreads();
        return;
    }
    const int nq = P.t.n[q], nq2 = nq * nq, nq3 = nq2 * nq;
    const double* A = B(P, P.bi.d2f[nq][n]);  // n x nq
    const int row = (fq & 1) ? n - 1 : 0;
    face_map_t(lb, n, sT1, nq, A, V, sT2);
    double* dst = Ub + P.t.off[q];
    for (int i = threadIdx.x; i < V * nq3; i += blockDim.x) {
        const int v = i / nq3, c = i % nq3;
        const int ii = c % nq, jj = (c / nq) % nq, kk = c / nq2;
        const int m = d == 0 ? ii : (d == 1 ? jj : kk);
        const int a = d == 0 ? jj : ii, b = d == 2 ? jj : kk;
        const double x = __ldg(A + row * nq + m) * sT1[v * nq2 + a + nq * b];
        if (ATOMIC) atomicAdd(dst + (int64_t)v * nq3 + c, x);
        else dst[(int64_t)v * nq3 + c] += x;
    }
    __syncthreads();
}

// A face that changes representation (Sec. 3.2.1, 3.2.2): the common
// representation and which side is mapped to it.  DG/DG: the higher degree,
// the lower side mapped.  DG/FV: the FV side's sub-cells, the DG side mapped
// (V^{DG->FV}).  FV/FV with different sub-cell counts (per-element counts):
// the finer grid, the coarser side mapped by its sub-cell overlaps.
struct MixedFace {
    int eL, eR, nc;
    bool cfv, mapL;
};

__device__ __forceinline__ MixedFace mixed_face(const Params& P, const Faces& Fc, int fid) {
    MixedFace m;
    m.eL = Fc.L[fid];
    m.eR = Fc.R[fid];
    const bool fL = P.t.fv[m.eL], fR = P.t.fv[m.eR];
    m.cfv = fL || fR;
    const int nL = P.t.n[m.eL], nR = P.t.n[m.eR];
    if (fL && fR) {
        m.nc = max(nL, nR);
        m.mapL = nL < nR;
    } else if (m.cfv) {
        m.nc = fL ? nL : nR;
        m.mapL = !fL;
    } else {
        m.nc = max(nL, nR);
        m.mapL = nL != m.nc;
    }
    return m;
}

}  // namespace dgfv
