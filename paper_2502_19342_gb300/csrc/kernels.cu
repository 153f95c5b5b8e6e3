// FP64 CUDA kernels of the hybrid DG/FV right-hand side (sm_103a).
//
// One stage R(U), in the paper's order of dependencies:
//   k_prolong    face values: DG traces u(+-1) (Sec. 3.1.1), FV boundary sub-cell means
//                (fused into the previous stage's k_surface within a step)
//   k_fv         FV sub-cell elements (Sec. 3.1.2): minmod reconstruction, central
//                gradients, interior sub-cell fluxes, element-face states (fv.cu)
//   k_face_lift* BR1 lifting value U* = (u- + u+)/2 (Eq. 19) on the lower degree /
//                on DG data at DG/FV faces (Sec. 3.2.2)
//   k_dg_volume  lifting (Eq. 23) -> gradient in shared memory -> fluxes at the nodes
//                -> volume integral (Eq. 22); traces of the gradient
//                (k_dg_volume_split: the split form on LGL nodes, Sec. 3.5; volume.cu)
//   k_face_flux_conf, k_mixed_*
//                F* = F^c* + (F^v- + F^v+)/2 (Eqs. 20, 21) on the higher degree / on
//                FV data (Sec. 3.2.1), mapped back to both sides
//   k_surface    surface integral and -1/J (Eqs. 22, 26), fused with the Runge-Kutta
//                stage update (k_pp_limit after it when the limiter is on)
// plus the time step (Sec. 3.3), the modal indicator (Sec. 3.4) and the remap
// of adapted elements (Sec. 3.2 mappings).
//
// The path is bound by the FP64 pipe: the kernels trade shared-memory traffic
// and integer work for fewer FP64 instructions (reciprocals computed once,
// sum-factorised contractions, fused multiply-adds).
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cstdint>
#include <mutex>

#include "common.cuh"
#include "device_util.cuh"
#include "kernels.h"

namespace dgfv {


// ---------------------------------------------------------------------------------
// Face values of a tile of elements whose states sit in shared memory
// (sU: count x V x n^3): u(+-1) = sum_m l_m(+-1) u_m along the face normal for DG
// elements, the boundary sub-cell mean for FV elements.  One thread per face
// point, all variables.
template <int NK, int NP = 0>
__device__ __forceinline__ void tile_face_values(const Params& P, const Tiles& T, int first, int count, int n_rt,
                                                 const double* sU, const double* sl) {
    constexpr int V = NK + 4;
    const int n = NP > 0 ? NP : n_rt;
    const int n2 = n * n, n3 = n2 * n, per = 6 * n2;
    for (int i = threadIdx.x; i < count * per; i += blockDim.x) {
        const int el = i / per, r = i - el * per, f = r / n2, p = r - f * n2;
        const int a = p % n, b = p / n, d = f >> 1, side = f & 1;
        const int e = T.items[first + el];
        const double* src = sU + el * V * n3;
        double* dst = P.b.fu + (P.t.fo[e] + (int64_t)f * n2) * V + p;
        if (P.t.fv[e]) {
            const int c = node_index(n, d, side ? n - 1 : 0, a, b);
#pragma unroll
            for (int v = 0; v < V; ++v) dst[v * n2] = src[v * n3 + c];
        } else {
            const double* l = sl + (side ? MAXP : 0);
            const int c0 = node_index(n, d, 0, a, b), st = d == 0 ? 1 : (d == 1 ? n : n2);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                double val = 0.0;
                for (int m = 0; m < n; ++m) val = fma(l[m], src[v * n3 + c0 + m * st], val);
                dst[v * n2] = val;
            }
        }
    }
}

// k_prolong: face values of every element (tile staged in shared memory).
template <int NK>
__global__ void __launch_bounds__(256) k_prolong(Params P, Tiles T, const double* __restrict__ U) {
    constexpr int V = NK + 4;
    extern __shared__ double sm[];
    double* sl = sm;              // lm, lp
    double* sU = sm + 2 * MAXP;   // count * V n^3
    const int first = T.first[blockIdx.x], count = T.count[blockIdx.x], n = T.n[blockIdx.x];
    const int n3 = n * n * n, per = V * n3;
    if (threadIdx.x < n) {
        sl[threadIdx.x] = B(P, P.bi.lm[n])[threadIdx.x];
        sl[MAXP + threadIdx.x] = B(P, P.bi.lp[n])[threadIdx.x];
    }
    for (int i = threadIdx.x; i < count * per; i += blockDim.x) {
        const int el = i / per, r = i - el * per;
        sU[i] = U[P.t.off[T.items[first + el]] + r];
    }
    __syncthreads();
    tile_face_values<NK>(P, T, first, count, n, sU, sl);
}

// ---------------------------------------------------------------------------------
// k_face_lift_conf: lifting value U* = (u- + u+)/2 on faces whose two sides are
// DG of one degree; one thread per face point (FV/FV faces of the conforming
// tiles carry no lifting value and are skipped).
__global__ void __launch_bounds__(128) k_face_lift_conf(Params P, Faces Fc, FaceTiles T, int V) {
    const int first = T.first[blockIdx.x], count = T.count[blockIdx.x], nc = T.nc[blockIdx.x], d = T.d[blockIdx.x];
    const int nc2 = nc * nc;
    for (int t = threadIdx.x; t < count * nc2; t += blockDim.x) {
        const int fid = T.items[first + t / nc2], p = t % nc2;
        const int eL = Fc.L[fid], eR = Fc.R[fid];
        if (P.t.fv[eL]) continue;
        const int64_t sL = (P.t.fo[eL] + (int64_t)(2 * d + 1) * nc2) * V + p;
        const int64_t sR = (P.t.fo[eR] + (int64_t)(2 * d) * nc2) * V + p;
        for (int v = 0; v < V; ++v) {
            const double u = 0.5 * (P.b.fu[sL + v * nc2] + P.b.fu[sR + v * nc2]);
            P.b.flift[sL + v * nc2] = u;
            P.b.flift[sR + v * nc2] = u;
        }
    }
}

// ---------------------------------------------------------------------------------
// k_face_lift: one CTA per face that has a DG side.
template <int NK>
__global__ void __launch_bounds__(64) k_face_lift(Params P, Faces Fc, const int32_t* __restrict__ list) {
    constexpr int V = NK + 4;
    __shared__ double sA[V * MAXP * MAXP], sB[V * MAXP * MAXP], sT[V * MAXP * MAXP];
    const int fid = list[blockIdx.x];
    const int eL = Fc.L[fid], eR = Fc.R[fid], d = Fc.d[fid];
    const int fL = 2 * d + 1, fR = 2 * d;
    const bool fvL = P.t.fv[eL], fvR = P.t.fv[eR];
    const int nL = P.t.n[eL], nR = P.t.n[eR];
    const int64_t sL = (P.t.fo[eL] + (int64_t)fL * nL * nL) * V;
    const int64_t sR = (P.t.fo[eR] + (int64_t)fR * nR * nR) * V;
    if (!fvL && !fvR) {
        if (nL == nR) {
            const int n2 = nL * nL;
            for (int i = threadIdx.x; i < V * n2; i += blockDim.x) {
                const double u = 0.5 * (P.b.fu[sL + i] + P.b.fu[sR + i]);
                P.b.flift[sL + i] = u;
                P.b.flift[sR + i] = u;
            }
            return;
        }
        // lifting on the lower degree m, interpolated back up (Sec. 3.2.2)
        const bool lowL = nL < nR;
        const int m = lowL ? nL : nR, M = lowL ? nR : nL;
        const int64_t sLo = lowL ? sL : sR, sHi = lowL ? sR : sL;
        for (int i = threadIdx.x; i < V * M * M; i += blockDim.x) sA[i] = P.b.fu[sHi + i];
        __syncthreads();
        face_map(sA, M, sB, m, B(P, P.bi.vm[M][m]), V, sT);  // L2 projection M -> m
        for (int i = threadIdx.x; i < V * m * m; i += blockDim.x) {
            const double u = 0.5 * (sB[i] + P.b.fu[sLo + i]);
            sB[i] = u;
            P.b.flift[sLo + i] = u;
        }
        __syncthreads();
        face_map(sB, m, sA, M, B(P, P.bi.vm[m][M]), V, sT);  // interpolation m -> M
        for (int i = threadIdx.x; i < V * M * M; i += blockDim.x) P.b.flift[sHi + i] = sA[i];
        return;
    }
    if (fvL && fvR) return;
    // DG/FV: FV face state mapped to the DG side's polynomial data by V^{FV->DG}
    const int nD = fvL ? nR : nL, nF = fvL ? nL : nR;
    const int64_t sD = fvL ? sR : sL, sF = fvL ? sL : sR;
    for (int i = threadIdx.x; i < V * nF * nF; i += blockDim.x) sA[i] = P.b.frec[sF + i];
    __syncthreads();
    face_map(sA, nF, sB, nD, B(P, P.bi.f2d[nD][nF]), V, sT);
    for (int i = threadIdx.x; i < V * nD * nD; i += blockDim.x) P.b.flift[sD + i] = 0.5 * (P.b.fu[sD + i] + sB[i]);
}

// ---------------------------------------------------------------------------------
// Face fluxes.  F* = F^c*(uL,uR) + (F^v(uL,gL) + F^v(uR,gR))/2 in +x_d, written as
// the outward flux of both sides (+F for the lower element, -F for the upper).
//
// k_face_flux_conf: faces whose two sides share one representation (equal DG
// degree, or FV on both sides); one thread per face point, operands straight
// from the face buffers, the direction a compile-time constant.
template <int NK, int D>
__device__ __forceinline__ void conf_face_body(const Params& P, const Faces& Fc, const int32_t* __restrict__ items,
                                               int first, int count, int nc) {
    constexpr int V = NK + 4;
    const int nc2 = nc * nc;
    const bool visc = P.ph.viscous;
    for (int t = threadIdx.x; t < count * nc2; t += blockDim.x) {
        const int fid = items[first + t / nc2], p = t % nc2;
        const int eL = Fc.L[fid], eR = Fc.R[fid];
        const int64_t sL = P.t.fo[eL] + (int64_t)(2 * D + 1) * nc2;
        const int64_t sR = P.t.fo[eR] + (int64_t)(2 * D) * nc2;
        const double* uLs = (P.t.fv[eL] ? P.b.frec : P.b.fu) + sL * V + p;
        const double* uRs = (P.t.fv[eR] ? P.b.frec : P.b.fu) + sR * V + p;
        double uL[V], uR[V], gL[3 * V], gR[3 * V], F[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            uL[v] = uLs[v * nc2];
            uR[v] = uRs[v * nc2];
        }
        if (visc) {
            const double* gLs = P.b.fg + sL * 3 * V + p;
            const double* gRs = P.b.fg + sR * 3 * V + p;
#pragma unroll
            for (int x = 0; x < 3 * V; ++x) {
                gL[x] = gLs[x * nc2];
                gR[x] = gRs[x * nc2];
            }
        }
        interface_flux<NK>(P.ph, uL, gL, uR, gR, D, F, P.t.fv[eL] != 0);  // conforming: both FV or both DG
        double* dL = P.b.flux + sL * V + p;
        double* dR = P.b.flux + sR * V + p;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            dL[v * nc2] = F[v];
            dR[v * nc2] = -F[v];
        }
    }
}

template <int NK>
__global__ void __launch_bounds__(128) k_face_flux_conf(Params P, Faces Fc, FaceTiles T) {
    const int first = T.first[blockIdx.x], count = T.count[blockIdx.x], nc = T.nc[blockIdx.x];
    switch (T.d[blockIdx.x]) {
        case 0: conf_face_body<NK, 0>(P, Fc, T.items, first, count, nc); break;
        case 1: conf_face_body<NK, 1>(P, Fc, T.items, first, count, nc); break;
        default: conf_face_body<NK, 2>(P, Fc, T.items, first, count, nc); break;
    }
}

// ---------------------------------------------------------------------------------
// Faces that change representation, in three passes (Sec. 3.2.1, 3.2.2): the
// side not in the common representation (always a DG side: the lower degree,
// or the DG side of a DG/FV face) is mapped to it (k_mixed_in: u and g by
// V^{N->Nc} or V^{DG->FV}, into scratch); the flux runs one thread per common
// face point like the conforming faces (k_mixed_flux; the other side read in
// place, its flux written directly); the mapped side's flux is mapped back
// (k_mixed_out: L2 projection or V^{FV->DG}).  Mixed face k: face mface[k],
// scratch at point offset mpt[k] (4V values per point in, V out).

template <int NK>
__global__ void __launch_bounds__(128) k_mixed_in(Params P, Faces Fc, const int32_t* __restrict__ mface,
                                                  const int64_t* __restrict__ mpt, double* __restrict__ Sin) {
    constexpr int V = NK + 4;
    __shared__ double tmp[3 * V * MAXP * MAXP];
    const int k = blockIdx.x, fid = mface[k], d = Fc.d[fid];
    const MixedFace m = mixed_face(P, Fc, fid);
    const int e = m.mapL ? m.eL : m.eR, f = m.mapL ? 2 * d + 1 : 2 * d, n = P.t.n[e];
    const int64_t slot = P.t.fo[e] + (int64_t)f * n * n;
    const bool fvs = P.t.fv[e];  // a coarser FV side (per-element counts): its reconstructed states by overlaps
    const double* M = B(P, fvs ? P.bi.ov[n][m.nc] : (m.cfv ? P.bi.d2f[n][m.nc] : P.bi.vm[n][m.nc]));
    double* out = Sin + mpt[k] * 4 * V;
    face_map((fvs ? P.b.frec : P.b.fu) + slot * V, n, out, m.nc, M, V, tmp);
    if (P.ph.viscous) face_map(P.b.fg + slot * 3 * V, n, out + V * m.nc * m.nc, m.nc, M, 3 * V, tmp);
}

template <int NK, int D>
__device__ __forceinline__ void mixed_flux_body(const Params& P, const Faces& Fc, const int32_t* __restrict__ mface,
                                                const int64_t* __restrict__ mpt, const double* __restrict__ Sin,
                                                double* __restrict__ Sout, const int32_t* __restrict__ items,
                                                int first, int count, int nc) {
    constexpr int V = NK + 4;
    const int nc2 = nc * nc;
    const bool visc = P.ph.viscous;
    for (int t = threadIdx.x; t < count * nc2; t += blockDim.x) {
        const int k = items[first + t / nc2], p = t % nc2;
        const MixedFace m = mixed_face(P, Fc, mface[k]);
        const int ed = m.mapL ? m.eR : m.eL, fd = m.mapL ? 2 * D : 2 * D + 1;
        const int64_t sd = P.t.fo[ed] + (int64_t)fd * nc2;
        const double* ud = (P.t.fv[ed] ? P.b.frec : P.b.fu) + sd * V + p;
        const double* gd = P.b.fg + sd * 3 * V + p;
        const double* um = Sin + mpt[k] * 4 * V + p;
        const double* gm = um + V * nc2;
        double uL[V], uR[V], gL[3 * V], gR[3 * V], F[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const double a = um[v * nc2], b = ud[v * nc2];
            uL[v] = m.mapL ? a : b;
            uR[v] = m.mapL ? b : a;
        }
        if (visc) {
#pragma unroll
            for (int x = 0; x < 3 * V; ++x) {
                const double a = gm[x * nc2], b = gd[x * nc2];
                gL[x] = m.mapL ? a : b;
                gR[x] = m.mapL ? b : a;
            }
        }
        interface_flux<NK>(P.ph, uL, gL, uR, gR, D, F, m.cfv);
        double* dd = P.b.flux + sd * V + p;
        double* so = Sout + mpt[k] * V + p;
        const double sgn = m.mapL ? -1.0 : 1.0;  // the direct side is the upper element when L is mapped
#pragma unroll
        for (int v = 0; v < V; ++v) {
            dd[v * nc2] = sgn * F[v];
            so[v * nc2] = F[v];
        }
    }
}

template <int NK>
__global__ void __launch_bounds__(128) k_mixed_flux(Params P, Faces Fc, FaceTiles T, const int32_t* __restrict__ mface,
                                                    const int64_t* __restrict__ mpt, const double* __restrict__ Sin,
                                                    double* __restrict__ Sout) {
    const int first = T.first[blockIdx.x], count = T.count[blockIdx.x], nc = T.nc[blockIdx.x];
    switch (T.d[blockIdx.x]) {
        case 0: mixed_flux_body<NK, 0>(P, Fc, mface, mpt, Sin, Sout, T.items, first, count, nc); break;
        case 1: mixed_flux_body<NK, 1>(P, Fc, mface, mpt, Sin, Sout, T.items, first, count, nc); break;
        default: mixed_flux_body<NK, 2>(P, Fc, mface, mpt, Sin, Sout, T.items, first, count, nc); break;
    }
}

template <int NK>
__global__ void __launch_bounds__(128) k_mixed_out(Params P, Faces Fc, const int32_t* __restrict__ mface,
                                                   const int64_t* __restrict__ mpt, const double* __restrict__ Sout) {
    constexpr int V = NK + 4;
    __shared__ double tmp[V * MAXP * MAXP], res[V * MAXP * MAXP];
    const int k = blockIdx.x, fid = mface[k], d = Fc.d[fid];
    const MixedFace m = mixed_face(P, Fc, fid);
    const int e = m.mapL ? m.eL : m.eR, f = m.mapL ? 2 * d + 1 : 2 * d, n = P.t.n[e], n2 = n * n;
    const double* M =
        B(P, P.t.fv[e] ? P.bi.ov[m.nc][n] : (m.cfv ? P.bi.f2d[n][m.nc] : P.bi.vm[m.nc][n]));
    face_map(Sout + mpt[k] * V, m.nc, res, n, M, V, tmp);
    const double sgn = m.mapL ? 1.0 : -1.0;  // outward normal of the upper element is -x_d
    double* dst = P.b.flux + (P.t.fo[e] + (int64_t)f * n2) * V;
    for (int i = threadIdx.x; i < V * n2; i += blockDim.x) dst[i] = sgn * res[i];
}

// ---------------------------------------------------------------------------------
// k_surface: surface integral and -1/J, fused with the Runge-Kutta stage update.
//   mode 0: out = R
//   mode 1: out = a*U0 + b*(Uin + dt*R)   (SSP-RK3; out may alias Uin or U0)
//   mode 2: dU = a*dU + dt*R; out = Uin + b*dU   (low-storage RK4; out may alias Uin)
// One thread per node, all variables.  With fuse != 0 (mode 1) the new state
// is also kept in shared memory and its face values are written for the next
// evaluation (the face-value pass of that evaluation is then skipped).
template <int NK, int MODE, int NP>
__device__ __forceinline__ void surface_body(const Params& P, const Tiles& T, const double* Uin, const double* U0,
                                             double* out, double a, double b, const double* __restrict__ dtp,
                                             int fuse, double* dU) {
    constexpr int mode = MODE;
    constexpr int V = NK + 4;
    extern __shared__ double sm[];
    double* sl = sm;             // lm, lp, lhm, lhp
    double* sU = sm + 4 * MAXP;  // count * V n^3 (fuse)
    const int first = T.first[blockIdx.x], count = T.count[blockIdx.x];
    const int n = NP > 0 ? NP : T.n[blockIdx.x];
    const int n2 = n * n, n3 = n2 * n;
    if (threadIdx.x < n) {
        sl[threadIdx.x] = B(P, P.bi.lm[n])[threadIdx.x];
        sl[MAXP + threadIdx.x] = B(P, P.bi.lp[n])[threadIdx.x];
        sl[2 * MAXP + threadIdx.x] = B(P, P.bi.lhm[n])[threadIdx.x];
        sl[3 * MAXP + threadIdx.x] = B(P, P.bi.lhp[n])[threadIdx.x];
    }
    __syncthreads();
    const double dt = mode ? *dtp : 0.0;
    for (int idx = threadIdx.x; idx < count * n3; idx += blockDim.x) {
        const int el = idx / n3, c = idx - el * n3;
        const int e = T.items[first + el];
        const int i = c % n, jk = c / n, j = jk % n, k = jk / n;
        const int m[3] = {i, j, k};
        const int pt[3] = {j + n * k, i + n * k, i + n * j};
        const int64_t off = P.t.off[e] + c, fo = P.t.fo[e];
        const bool fv = P.t.fv[e];
        // weights of the six face fluxes at this node (FV: boundary sub-cells only)
        double wm[3], wp[3];
        const double* Fm[3];
        const double* Fp[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double rh = P.t.rh[3 * e + d];
            if (fv) {
                const double sc = 0.5 * n * rh;  // n/h_d
                wm[d] = m[d] == 0 ? sc : 0.0;
                wp[d] = m[d] == n - 1 ? sc : 0.0;
            } else {
                wm[d] = rh * sl[2 * MAXP + m[d]];
                wp[d] = rh * sl[3 * MAXP + m[d]];
            }
            Fm[d] = P.b.flux + (fo + (int64_t)(2 * d) * n2) * V + pt[d];
            Fp[d] = P.b.flux + (fo + (int64_t)(2 * d + 1) * n2) * V + pt[d];
        }
        // new state of the node, for the positivity check: rho and 2 rho (rho e)
        double nrho = 0.0, nm2 = 0.0, nE = 0.0;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            double acc = P.b.rtmp[off + (int64_t)v * n3];
#pragma unroll
            for (int d = 0; d < 3; ++d) acc = fma(wp[d], Fp[d][v * n2], fma(wm[d], Fm[d][v * n2], acc));
            const double R = -acc;
            if (mode == 0) {
                out[off + (int64_t)v * n3] = R;
            } else {
                double x;
                if (mode == 1) {
                    // a = 0 (first stage): U0 is not read
                    const double y = fma(dt, R, Uin[off + (int64_t)v * n3]);
                    x = a == 0.0 ? b * y : fma(b, y, a * U0[off + (int64_t)v * n3]);
                } else {
                    // a = 0 (first stage): the previous dU is not read
                    const double y = a == 0.0 ? dt * R : fma(a, dU[off + (int64_t)v * n3], dt * R);
                    dU[off + (int64_t)v * n3] = y;
                    x = fma(b, y, Uin[off + (int64_t)v * n3]);
                }
                if (nonfinite_bits(x)) set_status(P.status, -5, e);
                if (v < NK) nrho += x;
                else if (v < NK + 3) nm2 = fma(x, x, nm2);
                else nE = x;
                out[off + (int64_t)v * n3] = x;
                if (fuse) sU[el * V * n3 + v * n3 + c] = x;
            }
        }
        // rho <= 0 or rho e = rho E - |rho v|^2/(2 rho) <= 0 (p <= 0, as kappa > 1);
        // false for NaN, which the non-finite check reports
        if (mode != 0 && (nrho <= 0.0 || fma(2.0 * nrho, nE, -nm2) <= 0.0)) set_status(P.status, -4, e);
    }
    if (fuse) {
        __syncthreads();
        tile_face_values<NK, NP>(P, T, first, count, n, sU, sl);
    }
}

// NP: the tile's point count as a compile-time constant.
template <int NK, int MODE>
__global__ void __launch_bounds__(256) k_surface(Params P, Tiles T, const double* Uin, const double* U0,
                                                 double* out, double a, double b,
                                                 const double* __restrict__ dtp, int fuse, double* dU) {
    switch (T.n[blockIdx.x]) {
        case 2: surface_body<NK, MODE, 2>(P, T, Uin, U0, out, a, b, dtp, fuse, dU); break;
        case 3: surface_body<NK, MODE, 3>(P, T, Uin, U0, out, a, b, dtp, fuse, dU); break;
        case 4: surface_body<NK, MODE, 4>(P, T, Uin, U0, out, a, b, dtp, fuse, dU); break;
        case 5: surface_body<NK, MODE, 5>(P, T, Uin, U0, out, a, b, dtp, fuse, dU); break;
        case 6: surface_body<NK, MODE, 6>(P, T, Uin, U0, out, a, b, dtp, fuse, dU); break;
        case 7: surface_body<NK, MODE, 7>(P, T, Uin, U0, out, a, b, dtp, fuse, dU); break;
        case 8: surface_body<NK, MODE, 8>(P, T, Uin, U0, out, a, b, dtp, fuse, dU); break;
        default: surface_body<NK, MODE, 0>(P, T, Uin, U0, out, a, b, dtp, fuse, dU); break;  // N_FV = 9
    }
}

// ---------------------------------------------------------------------------------
// k_pp_limit: Zhang-Shu positivity limiter (Sec. 3.5), one CTA per DG element.
// Element mean by the element's quadrature; check points = nodes + face points;
// (1) every partial density towards its mean (floor min(eps, mean));
// (2) one factor theta for all variables from the internal energy rho e =
//     rho E - |rho v|^2/(2 rho): at a check point below the floor, t solves the
//     quadratic rho(t) (rho E(t) - floor) - |m(t)|^2/2 = 0 on the segment from the
//     mean (closed form; rho e is concave along it, one root in (0, 1)).
// Changed elements are written back (state and their face values for the next
// stage) and counted.
template <int NK>
__global__ void __launch_bounds__(128) k_pp_limit(Params P, const int32_t* __restrict__ items, double* U,
                                                  double eps, unsigned long long* count, int write_faces) {
    constexpr int V = NK + 4;
    extern __shared__ double sm[];
    __shared__ double red[V][4];
    __shared__ double s_theta[NK + 1];
    __shared__ int s_active;
    const int e = items[blockIdx.x];
    const int n = P.t.n[e], n2 = n * n, n3 = n2 * n, nf = 6 * n2;
    double* su = sm;            // V * n3 nodes
    double* sf = su + V * n3;   // V * 6 n^2 face points
    double* sw = sf + V * nf;   // weights (n), lm, lp (n each)
    double* src = U + P.t.off[e];
    if (threadIdx.x < n) {
        sw[threadIdx.x] = B(P, P.bi.w[n])[threadIdx.x];
        sw[n + threadIdx.x] = B(P, P.bi.lm[n])[threadIdx.x];
        sw[2 * n + threadIdx.x] = B(P, P.bi.lp[n])[threadIdx.x];
    }
    if (threadIdx.x == 0) s_active = 0;
    for (int i = threadIdx.x; i < V * n3; i += blockDim.x) su[i] = src[i];
    __syncthreads();
    // element mean (fixed per-thread order, then a fixed reduction order)
    double part[V];
#pragma unroll
    for (int v = 0; v < V; ++v) part[v] = 0.0;
    for (int c = threadIdx.x; c < n3; c += blockDim.x) {
        const double w = sw[c % n] * sw[(c / n) % n] * sw[c / n2];
#pragma unroll
        for (int v = 0; v < V; ++v) part[v] = fma(w, su[v * n3 + c], part[v]);
    }
    __shared__ double sred[V][128 / 32];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        double x = part[v];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) sred[v][threadIdx.x >> 5] = x;
    }
    // face points
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
        const int f = i / n2, p = i % n2, d = f >> 1, a = p % n, b = p / n;
        const double* l = sw + ((f & 1) ? 2 * n : n);
        const int c0 = node_index(n, d, 0, a, b), st = d == 0 ? 1 : (d == 1 ? n : n2);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            double s = 0.0;
            for (int m = 0; m < n; ++m) s = fma(l[m], su[v * n3 + c0 + m * st], s);
            sf[v * nf + i] = s;
        }
    }
    __syncthreads();
    double mean[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        double x = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x += sred[v][w];
        mean[v] = 0.125 * x;
    }
    // (1) partial densities: minima over nodes and face points
    double mn[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) mn[k] = mean[k];
    for (int i = threadIdx.x; i < n3 + nf; i += blockDim.x) {
#pragma unroll
        for (int k = 0; k < NK; ++k) mn[k] = fmin(mn[k], i < n3 ? su[k * n3 + i] : sf[k * nf + i - n3]);
    }
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        double x = mn[k];
        for (int o = 16; o > 0; o >>= 1) x = fmin(x, __shfl_down_sync(0xffffffffu, x, o));
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            double x = red[k][0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) x = fmin(x, red[k][w]);
            const double ek = fmin(eps, mean[k]);
            s_theta[k] = x < ek ? (mean[k] - ek) / (mean[k] - x) : 1.0;
            if (x < ek) s_active = 1;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n3 + nf; i += blockDim.x) {
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            const double th = s_theta[k];
            if (th < 1.0) {
                double* q = i < n3 ? &su[k * n3 + i] : &sf[k * nf + i - n3];
                *q = fma(th, *q - mean[k], mean[k]);
            }
        }
    }
    __syncthreads();
    // (2) internal energy
    double rb = 0.0;
#pragma unroll
    for (int k = 0; k < NK; ++k) rb += mean[k];
    const double mb2 = mean[NK] * mean[NK] + mean[NK + 1] * mean[NK + 1] + mean[NK + 2] * mean[NK + 2];
    const double ee = fmin(eps, mean[NK + 3] - 0.5 * mb2 / rb);
    double tmin = 1.0;
    for (int i = threadIdx.x; i < n3 + nf; i += blockDim.x) {
        double q[V];
#pragma unroll
        for (int v = 0; v < V; ++v) q[v] = i < n3 ? su[v * n3 + i] : sf[v * nf + i - n3];
        double r = 0.0;
#pragma unroll
        for (int k = 0; k < NK; ++k) r += q[k];
        const double m2 = q[NK] * q[NK] + q[NK + 1] * q[NK + 1] + q[NK + 2] * q[NK + 2];
        if (q[NK + 3] - 0.5 * m2 / r >= ee) continue;
        double ar = 0.0;
#pragma unroll
        for (int k = 0; k < NK; ++k) ar += q[k] - mean[k];
        const double aE = q[NK + 3] - mean[NK + 3];
        double am2 = 0.0, mam = 0.0;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const double a = q[NK + j] - mean[NK + j];
            am2 = fma(a, a, am2);
            mam = fma(mean[NK + j], a, mam);
        }
        const double c0 = rb * (mean[NK + 3] - ee) - 0.5 * mb2;
        const double c1 = rb * aE + ar * (mean[NK + 3] - ee) - mam;
        const double c2 = ar * aE - 0.5 * am2;
        double t;
        if (fabs(c2) <= 1e-14 * (fabs(c1) + fabs(c0))) {
            t = -c0 / c1;
        } else {
            const double disc = fmax(c1 * c1 - 4.0 * c0 * c2, 0.0);
            const double qq = -0.5 * (c1 + copysign(sqrt(disc), c1));
            const double r1 = qq / c2, r2 = c0 / qq;
            t = 1.0;
            if (r1 >= 0.0 && r1 <= 1.0) t = fmin(t, r1);
            if (r2 >= 0.0 && r2 <= 1.0) t = fmin(t, r2);
        }
        tmin = fmin(tmin, fmax(t, 0.0));
    }
    for (int o = 16; o > 0; o >>= 1) tmin = fmin(tmin, __shfl_down_sync(0xffffffffu, tmin, o));
    if ((threadIdx.x & 31) == 0) red[0][threadIdx.x >> 5] = tmin;
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = red[0][0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) x = fmin(x, red[0][w]);
        s_theta[NK] = x;
        if (x < 1.0) s_active = 1;
        if (s_active) atomicAdd(count, 1ULL);
    }
    __syncthreads();
    if (!s_active) return;
    const double th = s_theta[NK];
    for (int i = threadIdx.x; i < V * n3; i += blockDim.x) {
        const int v = i / n3;
        src[i] = th < 1.0 ? fma(th, su[i] - mean[v], mean[v]) : su[i];
    }
    if (write_faces) {
        for (int i = threadIdx.x; i < V * nf; i += blockDim.x) {
            const int v = i / nf, r = i % nf, f = r / n2, p = r % n2;
            const double x = th < 1.0 ? fma(th, sf[i] - mean[v], mean[v]) : sf[i];
            P.b.fu[(P.t.fo[e] + (int64_t)f * n2) * V + v * n2 + p] = x;
        }
    }
}

// ---------------------------------------------------------------------------------
// Time step of Sec. 3.3: per-block maxima of the inverse time scales
//   lc = (2N+1) sum_d (|v_d| + c)/dx_d,  lv = (2N+1) dv sum_d 1/dx_d^2
// (FV: factor 1, dx = h/N_FV), then dt_c = cfl_c / max lc and dt_v = cfl_v / max lv
// in a final reduction (identical to the minimum of the per-node quotients,
// since correctly rounded division is monotone).  One reciprocal per node:
// with r = 1/(rho (rho c_v)(rho Pr)), 1/rho, 1/(rho c_v) and 1/(rho Pr) are products.
template <int NK>
__global__ void __launch_bounds__(256) k_dt(Params P, Tiles T, const double* __restrict__ U,
                                            double* __restrict__ partial) {
    constexpr int V = NK + 4;
    __shared__ double red[2][256 / 32];
    const int first = T.first[blockIdx.x], count = T.count[blockIdx.x], n = T.n[blockIdx.x];
    const int n3 = n * n * n;
    const bool visc = P.ph.viscous;
    double mc = 0.0, mv = 0.0, kc[3] = {0.0, 0.0, 0.0}, kv = 0.0;
    int ce = -1;
    for (int idx = threadIdx.x; idx < count * n3; idx += blockDim.x) {
        const int el = idx / n3, c = idx - el * n3;
        const int e = T.items[first + el];
        const double* src = U + P.t.off[e] + c;
        double u[V];
#pragma unroll
        for (int v = 0; v < V; ++v) u[v] = src[(int64_t)v * n3];
        double rho = u[0], rcv = 0.0, rcp = 0.0, rmu = 0.0, rpr = 0.0;
#pragma unroll
        for (int k = 1; k < NK; ++k) rho += u[k];
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            rcv = fma(u[k], P.ph.cv[k], rcv);
            rcp = fma(u[k], P.ph.cp[k], rcp);
            rmu = fma(u[k], P.ph.mu[k], rmu);
            rpr = fma(u[k], P.ph.pr[k], rpr);
        }
        const double t = rcv * rpr, r = 1.0 / (rho * t);
        const double irho = t * r, ircv = (rho * rpr) * r;
        double vv[3], ke = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            vv[d] = u[NK + d] * irho;
            ke = fma(vv[d], vv[d], ke);
        }
        const double eps = fma(-0.5, ke, u[NK + 3] * irho);
        const double cs = sqrt(rcp * (rcp - rcv) * eps) * ircv;  // c^2 = c_p (c_p - c_v) eps / c_v^2
        if (e != ce) {  // per-element constants: (2N+1)/dx_d and (2N+1) sum_d 1/dx_d^2
            ce = e;
            const bool fv = P.t.fv[e];
            const double fac = fv ? 1.0 : 2.0 * P.t.N[e] + 1.0;
            const double sub = fv ? (double)P.t.n[e] : 1.0;
            double sdx = 0.0;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const double idx_d = 0.5 * P.t.rh[3 * e + d] * sub;  // 1/dx_d
                kc[d] = idx_d * fac;
                sdx = fma(idx_d, idx_d, sdx);
            }
            kv = sdx * fac;
        }
        const double lam = fma(fabs(vv[0]) + cs, kc[0], fma(fabs(vv[1]) + cs, kc[1], (fabs(vv[2]) + cs) * kc[2]));
        mc = fmax(mc, lam);
        if (visc) {
            const double irpr = (rho * rcv) * r;
            if (P.ph.sutherland) rmu *= sutherland_factor(P.ph, eps * rho * ircv);  // T = eps / c_v
            // max(4/3 mu/rho, kappa mu/(Pr rho), max_k D_k)
            double dv = fmax(4.0 / 3.0 * rmu * irho * irho, rcp * rmu * ircv * irpr * irho);
            dv = fmax(dv, P.ph.maxD);
            mv = fmax(mv, dv * kv);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        mc = fmax(mc, __shfl_down_sync(0xffffffffu, mc, o));
        mv = fmax(mv, __shfl_down_sync(0xffffffffu, mv, o));
    }
    const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
    if (ln == 0) { red[0][w] = mc; red[1][w] = mv; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) { mc = fmax(mc, red[0][i]); mv = fmax(mv, red[1][i]); }
        partial[2 * blockIdx.x] = mc;
        partial[2 * blockIdx.x + 1] = mv;
    }
}

__global__ void k_dt_final(const double* __restrict__ partial, int nb, int viscous, double cfl_c, double cfl_v,
                           double* __restrict__ out3) {
    __shared__ double red[2][32];
    double mc = 0.0, mv = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        mc = fmax(mc, partial[2 * i]);
        mv = fmax(mv, partial[2 * i + 1]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        mc = fmax(mc, __shfl_down_sync(0xffffffffu, mc, o));
        mv = fmax(mv, __shfl_down_sync(0xffffffffu, mv, o));
    }
    const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
    if (ln == 0) { red[0][w] = mc; red[1][w] = mv; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) { mc = fmax(mc, red[0][i]); mv = fmax(mv, red[1][i]); }
        const double dtc = cfl_c / mc, dtv = viscous ? cfl_v / mv : INFINITY;
        out3[1] = dtc;
        out3[2] = dtv;
        out3[0] = viscous ? 1.0 / (1.0 / dtc + 1.0 / dtv) : dtc;
    }
}

__global__ void k_set_scalar(double* p, double v) { *p = v; }

// Copy of n doubles by every thread of a grid-stride loop, 16 bytes per
// access (both pointers 16-byte aligned; the odd last element by thread 0),
// for the state copies between device memory and page-locked host memory
// seen through its device mapping.
__global__ void __launch_bounds__(256) k_copy_state2(double* __restrict__ dst, const double* __restrict__ src,
                                                     int64_t n) {
    const int64_t n2 = n >> 1;
    double2* d2 = reinterpret_cast<double2*>(dst);
    const double2* s2 = reinterpret_cast<const double2*>(src);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x)
        d2[i] = s2[i];
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) dst[n - 1] = src[n - 1];
}

// The same, 8 bytes per access (a pointer not 16-byte aligned).
__global__ void __launch_bounds__(256) k_copy_state1(double* __restrict__ dst, const double* __restrict__ src,
                                                     int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// Decision thresholds of Sec. 3.4: FV on / FV off (on I_h), refine / coarsen (on I_rho).
struct Thresholds {
    double fv_on, fv_off, ref, crs;
};

// ---------------------------------------------------------------------------------
// Modal indicator (Sec. 3.4): one CTA per element.
template <int NK>
__global__ void __launch_bounds__(128) k_indicator(Params P, const double* __restrict__ U, int n_elem,
                                                   double* Ip, double* Ih, uint8_t* dec, Thresholds thr,
                                                   int N_min, int N_max, int vars, int P3) {
    // P3: scratch stride, the cube of the context's largest point count
    constexpr int V = NK + 4, NQ = 2 + (NK - 1);  // rho, p, Y_1..Y_{NK-1}
    extern __shared__ double sm[];
    double* sMap = sm;               // V*P3: FV state mapped to the element's degree
    double* sS1 = sMap + V * P3;     // P3 scratch
    double* sS2 = sS1 + P3;          // P3 scratch
    double* sQ = sS2 + P3;           // NQ*P3
    double* sQ2 = sQ + NQ * P3;      // NQ*P3
    __shared__ double sE[NQ][3][MAXP];
    __shared__ double sI[NQ][3];
    const int e = blockIdx.x;
    if (e >= n_elem) return;
    const int N = P.t.N[e], n = N + 1, n2 = n * n, n3 = n2 * n;
    const bool fv = P.t.fv[e];
    const double* src = U + P.t.off[e];
    if (fv) {
        // V^{FV->DG} in three directions, one variable at a time
        const int nf = P.t.n[e], nf2 = nf * nf, nf3 = nf2 * nf;
        const double* X = B(P, P.bi.f2d[n][nf]);  // n x nf
        for (int v = 0; v < V; ++v) {
            for (int idx = threadIdx.x; idx < n * nf2; idx += blockDim.x) {
                const int i = idx % n, jk = idx / n;
                double s = 0.0;
                for (int m = 0; m < nf; ++m) s = fma(__ldg(X + i * nf + m), src[(int64_t)v * nf3 + m + nf * jk], s);
                sS1[idx] = s;  // [i + n*(j + nf*k)]
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < n2 * nf; idx += blockDim.x) {
                const int i = idx % n, j = (idx / n) % n, k = idx / n2;
                double s = 0.0;
                for (int m = 0; m < nf; ++m) s = fma(__ldg(X + j * nf + m), sS1[i + n * (m + nf * k)], s);
                sS2[idx] = s;  // [i + n*(j + n*k)]
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < n3; idx += blockDim.x) {
                const int ij = idx % n2, k = idx / n2;
                double s = 0.0;
                for (int m = 0; m < nf; ++m) s = fma(__ldg(X + k * nf + m), sS2[ij + n2 * m], s);
                sMap[v * n3 + idx] = s;
            }
            __syncthreads();
        }
    }
    // quantities at the nodes
    for (int c = threadIdx.x; c < n3; c += blockDim.x) {
        double u[V];
        if (fv) {
#pragma unroll
            for (int v = 0; v < V; ++v) u[v] = sMap[v * n3 + c];
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) u[v] = src[(int64_t)v * n3 + c];
        }
        Prim<NK> s;
        prim<NK>(P.ph, u, s);
        sQ2[0 * n3 + c] = s.rho;
        sQ2[1 * n3 + c] = s.p;
#pragma unroll
        for (int k = 0; k + 1 < NK; ++k) sQ2[(2 + k) * n3 + c] = s.Y[k];
    }
    __syncthreads();
    // Legendre coefficients: three passes of the inverse Vandermonde
    const double* Vi = B(P, P.bi.vinv[n]);
    for (int idx = threadIdx.x; idx < NQ * n3; idx += blockDim.x) {
        const int q = idx / n3, c = idx % n3, i = c % n, jk = c / n;
        double s = 0.0;
        for (int m = 0; m < n; ++m) s = fma(__ldg(Vi + i * n + m), sQ2[q * n3 + m + n * jk], s);
        sQ[idx] = s;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < NQ * n3; idx += blockDim.x) {
        const int q = idx / n3, c = idx % n3, i = c % n, j = (c / n) % n, k = c / n2;
        double s = 0.0;
        for (int m = 0; m < n; ++m) s = fma(__ldg(Vi + j * n + m), sQ[q * n3 + i + n * (m + n * k)], s);
        sQ2[idx] = s;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < NQ * n3; idx += blockDim.x) {
        const int q = idx / n3, c = idx % n3, ij = c % n2, k = c / n2;
        double s = 0.0;
        for (int m = 0; m < n; ++m) s = fma(__ldg(Vi + k * n + m), sQ2[q * n3 + ij + n2 * m], s);
        sQ[idx] = s;
    }
    __syncthreads();
    // directional modal energies (fixed summation order per entry)
    for (int idx = threadIdx.x; idx < NQ * 3 * n; idx += blockDim.x) {
        const int q = idx / (3 * n), d = (idx / n) % 3, m = idx % n;
        double E = 0.0;
        for (int b = 0; b < n; ++b)
            for (int a = 0; a < n; ++a) {
                const double c = sQ[q * n3 + node_index(n, d, m, a, b)];
                E = fma(c, c, E);
            }
        sE[q][d][m] = E;
    }
    __syncthreads();
    // least-squares decay rate per direction (Eq. 34), I = min_d |sigma_d| (Eq. 35)
    for (int idx = threadIdx.x; idx < NQ * 3; idx += blockDim.x) {
        const int q = idx / 3, d = idx % 3;
        double total = 0.0;
        for (int m = 0; m < n; ++m) total += sE[q][0][m];
        double y[MAXP];
        double ybar = 0.0;
        for (int m = 0; m < n; ++m) {
            const double w = total > 0.0 ? sE[q][d][m] / total : 0.0;
            y[m] = log(fmax(w, 1e-24));  // energy fractions below 1e-24 are FP64 round-off
            ybar += y[m];
        }
        ybar /= n;
        const double mbar = 0.5 * (n - 1);
        double sxy = 0.0, sxx = 0.0;
        for (int m = 0; m < n; ++m) {
            sxy += (m - mbar) * (y[m] - ybar);
            sxx += (m - mbar) * (m - mbar);
        }
        sI[q][d] = fabs(sxy / sxx);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double I[NQ];
        for (int q = 0; q < NQ; ++q) I[q] = fmin(sI[q][0], fmin(sI[q][1], sI[q][2]));
        double ip = I[0], ih = I[1];
        for (int q = 2; q < NQ; ++q) ih = fmin(ih, I[q]);
        if (vars == 1) {  // p-refinement on I(p), FV on I(rho) (Sec. 4.3)
            ip = I[1];
            ih = I[0];
        }
        if (Ip) Ip[e] = ip;
        if (Ih) Ih[e] = ih;
        uint8_t code = 0;
        if (fv) {
            if (ih > thr.fv_off) code = 2;
        } else if (ih < thr.fv_on) {
            code = 1;
        } else if (ip < thr.ref && N < N_max) {
            code = 3;
        } else if (ip > thr.crs && N > N_min) {
            code = 4;
        }
        if (dec) dec[e] = code;
    }
}

// ---------------------------------------------------------------------------------
// Remap of the state to a new degree / FV pattern: one CTA per element.
struct RemapSide {
    const uint8_t* n;
    const uint8_t* N;
    const uint8_t* fv;
    const int64_t* off;
};

__global__ void __launch_bounds__(128) k_remap(Params P, RemapSide A, RemapSide Bn, int V, const double* __restrict__ Uo,
                                               double* __restrict__ Un) {
    extern __shared__ double sm[];
    const int e = blockIdx.x;
    const int na = A.n[e], nb = Bn.n[e];
    const bool fa = A.fv[e], fb = Bn.fv[e];
    const double* src = Uo + A.off[e];
    double* dst = Un + Bn.off[e];
    if (fa == fb && na == nb) {
        for (int i = threadIdx.x; i < V * na * na * na; i += blockDim.x) dst[i] = src[i];
        return;
    }
    const double* M;
    if (!fa && !fb) M = B(P, P.bi.vm[na][nb]);
    else if (!fa && fb) M = B(P, P.bi.d2f[na][nb]);
    else if (fa && !fb) M = B(P, P.bi.f2d[nb][na]);
    else M = B(P, P.bi.ov[na][nb]);  // FV -> FV with another sub-cell count (per-element counts)
    const int a2 = na * na, a3 = a2 * na, b2 = nb * nb, b3 = b2 * nb;
    double* t1 = sm;                 // V * nb*na*na
    double* t2 = t1 + V * nb * a2;   // V * nb*nb*na
    for (int idx = threadIdx.x; idx < V * nb * a2; idx += blockDim.x) {
        const int v = idx / (nb * a2), r = idx % (nb * a2), i = r % nb, jk = r / nb;
        double s = 0.0;
        for (int m = 0; m < na; ++m) s = fma(__ldg(M + i * na + m), src[(int64_t)v * a3 + m + na * jk], s);
        t1[idx] = s;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < V * b2 * na; idx += blockDim.x) {
        const int v = idx / (b2 * na), r = idx % (b2 * na), i = r % nb, j = (r / nb) % nb, k = r / b2;
        double s = 0.0;
        for (int m = 0; m < na; ++m) s = fma(__ldg(M + j * na + m), t1[v * nb * a2 + i + nb * (m + na * k)], s);
        t2[idx] = s;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < V * b3; idx += blockDim.x) {
        const int v = idx / b3, r = idx % b3, ij = r % b2, k = r / b2;
        double s = 0.0;
        for (int m = 0; m < na; ++m) s = fma(__ldg(M + k * na + m), t2[v * b2 * na + ij + b2 * m], s);
        dst[(int64_t)v * b3 + r] = s;
    }
}

// ---------------------------------------------------------------------------------
// FP64 peak probe: independent DFMA chains (8 per thread), no memory traffic.
__global__ void k_probe_dfma(int iters, double* sink) {
    double a0 = threadIdx.x * 1e-9, a1 = a0 + 1e-9, a2 = a0 + 2e-9, a3 = a0 + 3e-9;
    double a4 = a0 + 4e-9, a5 = a0 + 5e-9, a6 = a0 + 6e-9, a7 = a0 + 7e-9;
    const double x = 0.999999999, y = 1e-12;
    for (int i = 0; i < iters; ++i) {
        a0 = fma(a0, x, y); a1 = fma(a1, x, y); a2 = fma(a2, x, y); a3 = fma(a3, x, y);
        a4 = fma(a4, x, y); a5 = fma(a5, x, y); a6 = fma(a6, x, y); a7 = fma(a7, x, y);
    }
    const double s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
    if (s == 12345.0) sink[threadIdx.x] = s;
}

// FP64 tensor-core probe: eight independent mma.sync m8n8k4 (f64) accumulators
// per warp; each instruction is 8 x 8 x 4 FMAs.  Every lane of a warp runs it
// (all lanes converged), operands in registers only.
__global__ void k_probe_dmma(int iters, double* sink) {
    double c[8][2];
#pragma unroll
    for (int j = 0; j < 8; ++j) c[j][0] = c[j][1] = threadIdx.x * 1e-9 + j;
    const double a = 0.999999999, b = 1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                         : "+d"(c[j][0]), "+d"(c[j][1])
                         : "d"(a), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += c[j][0] + c[j][1];
    if (s == 12345.0) sink[threadIdx.x] = s;
}

// ================================================================= launchers
// ---------------------------------------------------------------------------------
// Non-conforming interfaces (Sec. 3.2.3).  Per direction of the big face: the
// map of half h, or the identity when the face is not halved that way.  On the
// big side's representation: DG nodes (n points) or FV sub-cells (fv).
__device__ __forceinline__ const double* mortar_dir(const Params& P, int split, int quad, int dir, bool fv, int n,
                                                    bool proj) {
    if (!((split >> dir) & 1)) return B(P, P.bi.eye[n]);
    const int h = (quad >> dir) & 1;
    if (fv) return B(P, proj ? P.bi.mfp[h] : P.bi.mfi[h]);
    return B(P, proj ? P.bi.mp[n][h] : P.bi.mi[n][h]);
}

// k_mortar_in: one CTA per virtual small side.  pass 0: the big side's face
// values interpolated to the quadrant (DG: the trace of u; FV: the
// reconstructed face state and, viscous, the boundary-cell gradient), after the
// FV kernel.  pass 1: the DG big side's gradient trace, after the volume kernel.
template <int NK>
__global__ void __launch_bounds__(128) k_mortar_in(Params P, MortarTables M, int pass) {
    constexpr int V = NK + 4;
    __shared__ double tmp[3 * V * MAXP * MAXP];
    const int v = M.n_elem + blockIdx.x, m = M.vmort[blockIdx.x], q = M.vquad[blockIdx.x];
    const int eb = M.big[m], fB = M.fB[m], sp = M.split[m];
    const bool fv = P.t.fv[eb];
    const int n = P.t.n[eb], n2 = n * n;
    if (pass == 1 && fv) return;
    const double* Ma = mortar_dir(P, sp, q, 0, fv, n, false);
    const double* Mb = mortar_dir(P, sp, q, 1, fv, n, false);
    const int64_t src = P.t.fo[eb] + (int64_t)fB * n2, dst = P.t.fo[v] + (int64_t)fB * n2;
    if (pass == 0) {
        const double* u = fv ? P.b.frec : P.b.fu;
        double* o = fv ? P.b.frec : P.b.fu;
        face_map2(u + src * V, n, o + dst * V, n, Ma, Mb, V, tmp);
        if (!fv || !P.ph.viscous) return;
    }
    face_map2(P.b.fg + src * 3 * V, n, P.b.fg + dst * 3 * V, n, Ma, Mb, 3 * V, tmp);
}

// k_mortar_out: one CTA per mortar; the L2 projection of the virtual sides'
// lifting values (which = 0, DG big sides) or outward fluxes (which = 1) onto
// the big side: F_0 = M_10 F_1 + M_20 F_2 (+ the other direction's halves).
template <int NK>
__global__ void __launch_bounds__(128) k_mortar_out(Params P, MortarTables M, int which) {
    constexpr int V = NK + 4;
    __shared__ double tmp[V * MAXP * MAXP], res[V * MAXP * MAXP], acc[V * MAXP * MAXP];
    const int m = blockIdx.x, eb = M.big[m], fB = M.fB[m], sp = M.split[m];
    const bool fv = P.t.fv[eb];
    if (which == 0 && fv) return;
    const int n = P.t.n[eb], n2 = n * n;
    double* buf = which == 0 ? P.b.flift : P.b.flux;
    for (int i = threadIdx.x; i < V * n2; i += blockDim.x) acc[i] = 0.0;
    for (int vi = M.vfirst[m]; vi < M.vfirst[m + 1]; ++vi) {
        const int v = M.n_elem + vi, q = M.vquad[vi];
        const double* Pa = mortar_dir(P, sp, q, 0, fv, n, true);
        const double* Pb = mortar_dir(P, sp, q, 1, fv, n, true);
        face_map2(buf + (P.t.fo[v] + (int64_t)fB * n2) * V, n, res, n, Pa, Pb, V, tmp);
        for (int i = threadIdx.x; i < V * n2; i += blockDim.x) acc[i] += res[i];
        __syncthreads();
    }
    double* dst = buf + (P.t.fo[eb] + (int64_t)fB * n2) * V;
    for (int i = threadIdx.x; i < V * n2; i += blockDim.x) dst[i] = acc[i];
}

// k_mortar_nb: one CTA per mortar face of an FV element: its neighbour values
// for the reconstruction and the central differences.  A small side takes the
// big element's layer on its quadrant (M^FV_01, M^FV_02); a big side the small
// elements' layers projected onto its sub-cells (M^FV_10, M^FV_20).
template <int NK>
__global__ void __launch_bounds__(128) k_mortar_nb(Params P, MortarTables M, const int32_t* __restrict__ active,
                                                   const double* __restrict__ U, double* __restrict__ out) {
    constexpr int V = NK + 4;
    __shared__ double sL[V * MAXP * MAXP], sR[V * MAXP * MAXP], sT1[V * MAXP * MAXP], sT2[V * MAXP * MAXP];
    const int sl = active[blockIdx.x], m = M.smort[sl], q = M.squad[sl], f = M.sface[sl];
    const int sp = M.split[m], n = P.nfv, n2 = n * n;
    double* dst = out + (int64_t)sl * V * n2;
    if (q >= 0) {
        const int eb = M.big[m];
        fv_layer<NK>(P, U, eb, M.fB[m], n, sL, sT1, sT2);
        face_map2(sL, n, dst, n, mortar_dir(P, sp, q, 0, true, n, false), mortar_dir(P, sp, q, 1, true, n, false), V,
                  sT1);
        return;
    }
    for (int i = threadIdx.x; i < V * n2; i += blockDim.x) dst[i] = 0.0;
    for (int vi = M.vfirst[m]; vi < M.vfirst[m + 1]; ++vi) {
        const int qq = M.vquad[vi];
        fv_layer<NK>(P, U, M.vsmall[vi], f ^ 1, n, sL, sT1, sT2);
        face_map2(sL, n, sR, n, mortar_dir(P, sp, qq, 0, true, n, true), mortar_dir(P, sp, qq, 1, true, n, true), V,
                  sT1);
        for (int i = threadIdx.x; i < V * n2; i += blockDim.x) dst[i] += sR[i];
        __syncthreads();
    }
}

#define DGFV_DISPATCH(nk, call)           \
    switch (nk) {                         \
        case 1: { constexpr int NK = 1; call; } break; \
        case 2: { constexpr int NK = 2; call; } break; \
        default: { constexpr int NK = 3; call; } break; \
    }

// Shared memory of the tile kernels that stage a tile of states: count * n^3 <= 512
// nodes per tile (the "all" tiling; an FV element of N_FV^3 > 512 sub-cells is a
// tile of its own) and 4 * MAXP bank values.
static size_t tile_state_smem(int nk, int nfv) {
    return sizeof(double) * (size_t)(4 * MAXP + (nk + 4) * std::max(512, nfv * nfv * nfv));
}

void launch_prolong(int nk, const Params& P, const Tiles& T, int ntiles, const double* U, cudaStream_t s) {
    if (ntiles <= 0) return;
    DGFV_DISPATCH(nk, (k_prolong<NK><<<ntiles, 256, tile_state_smem(nk, P.nfv), s>>>(P, T, U)));
}

void launch_face_lift_conf(int nk, const Params& P, const Faces& F, const FaceTiles& T, int ntiles, cudaStream_t s) {
    if (ntiles <= 0) return;
    k_face_lift_conf<<<ntiles, 128, 0, s>>>(P, F, T, nk + 4);
}

void launch_face_lift(int nk, const Params& P, const Faces& F, const int32_t* list, int nfaces, cudaStream_t s) {
    if (nfaces <= 0) return;
    DGFV_DISPATCH(nk, (k_face_lift<NK><<<nfaces, 64, 0, s>>>(P, F, list)));
}

void launch_mixed_faces(int nk, const Params& P, const Faces& F, const FaceTiles& T, int ntiles, const int32_t* mface,
                        const int64_t* mpt, int nmixed, double* Sin, double* Sout, cudaStream_t s) {
    if (nmixed <= 0) return;
    DGFV_DISPATCH(nk, (k_mixed_in<NK><<<nmixed, 128, 0, s>>>(P, F, mface, mpt, Sin),
                       k_mixed_flux<NK><<<ntiles, 128, 0, s>>>(P, F, T, mface, mpt, Sin, Sout),
                       k_mixed_out<NK><<<nmixed, 128, 0, s>>>(P, F, mface, mpt, Sout)));
}

void launch_mortar_in(int nk, const Params& P, const MortarTables& M, int n_virt, int pass, cudaStream_t s) {
    if (n_virt <= 0) return;
    DGFV_DISPATCH(nk, (k_mortar_in<NK><<<n_virt, 128, 0, s>>>(P, M, pass)));
}

void launch_mortar_out(int nk, const Params& P, const MortarTables& M, int n_mort, int which, cudaStream_t s) {
    if (n_mort <= 0) return;
    DGFV_DISPATCH(nk, (k_mortar_out<NK><<<n_mort, 128, 0, s>>>(P, M, which)));
}

void launch_mortar_nb(int nk, const Params& P, const MortarTables& M, const int32_t* active, int n_active,
                      const double* U, double* out, cudaStream_t s) {
    if (n_active <= 0) return;
    DGFV_DISPATCH(nk, (k_mortar_nb<NK><<<n_active, 128, 0, s>>>(P, M, active, U, out)));
}

void launch_face_flux_conf(int nk, const Params& P, const Faces& F, const FaceTiles& T, int ntiles, cudaStream_t s) {
    if (ntiles <= 0) return;
    DGFV_DISPATCH(nk, (k_face_flux_conf<NK><<<ntiles, 128, 0, s>>>(P, F, T)));
}

void launch_surface(int nk, const Params& P, const Tiles& T, int ntiles, const double* Uin, const double* U0,
                    double* out, int mode, double a, double b, const double* dt, bool fuse, double* dU,
                    cudaStream_t s) {
    if (ntiles <= 0) return;
    const int f = (fuse && mode != 0) ? 1 : 0;
    const size_t sm = f ? tile_state_smem(nk, P.nfv) : sizeof(double) * 4 * MAXP;
    if (mode == 0) {
        DGFV_DISPATCH(nk, (k_surface<NK, 0><<<ntiles, 256, sm, s>>>(P, T, Uin, U0, out, a, b, dt, f, dU)));
    } else if (mode == 1) {
        DGFV_DISPATCH(nk, (k_surface<NK, 1><<<ntiles, 256, sm, s>>>(P, T, Uin, U0, out, a, b, dt, f, dU)));
    } else {
        DGFV_DISPATCH(nk, (k_surface<NK, 2><<<ntiles, 256, sm, s>>>(P, T, Uin, U0, out, a, b, dt, f, dU)));
    }
}

void launch_dt(int nk, const Params& P, const Tiles& T, int ntiles, const double* U, double cfl_c, double cfl_v,
               double* partial, double* out3, cudaStream_t s) {
    DGFV_DISPATCH(nk, (k_dt<NK><<<ntiles, 256, 0, s>>>(P, T, U, partial)));
    k_dt_final<<<1, 1024, 0, s>>>(partial, ntiles, P.ph.viscous, cfl_c, cfl_v, out3);
}

void launch_set_scalar(double* p, double v, cudaStream_t s) { k_set_scalar<<<1, 1, 0, s>>>(p, v); }

void launch_copy_state(double* dst, const double* src, int64_t n, int n_sm, cudaStream_t s) {
    if (n <= 0) return;
    const int64_t per = ((((uintptr_t)dst | (uintptr_t)src) & 15) == 0) ? 2 : 1;
    const int64_t need = (n / per + 255) / 256;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)n_sm * 8));
    if (per == 2)
        k_copy_state2<<<blocks, 256, 0, s>>>(dst, src, n);
    else
        k_copy_state1<<<blocks, 256, 0, s>>>(dst, src, n);
}

void launch_pp_limit(int nk, const Params& P, const int32_t* items, int n_dg, double* U, double eps,
                     unsigned long long* count, bool write_faces, cudaStream_t s) {
    if (n_dg <= 0) return;
    const int V = nk + 4;
    const size_t sm = sizeof(double) * (size_t)(V * MAXP * MAXP * MAXP + 6 * V * MAXP * MAXP + 3 * MAXP);
    DGFV_DISPATCH(nk, (cudaFuncSetAttribute(k_pp_limit<NK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                       k_pp_limit<NK><<<n_dg, 128, sm, s>>>(P, items, U, eps, count, write_faces ? 1 : 0)));
}

// Scratch of the allocation-free time step (dgfv_compute_dt_noalloc): the
// per-block maxima of k_dt live in this fixed array instead of a buffer the
// context allocated.  Every device that loads the library holds the array
// (2 * DT_NOALLOC_MAX_BLOCKS doubles = 1 MiB) until the process exits.
static __device__ __align__(256) double g_dt_partial[2 * DT_NOALLOC_MAX_BLOCKS];

namespace {
std::mutex g_dt_partial_mutex;
double* g_dt_partial_addr[DT_NOALLOC_MAX_DEVICES] = {};
}  // namespace

int launch_dt_noalloc(int nk, const Params& P, const Tiles& T, int ntiles, const double* U, double cfl_c,
                      double cfl_v, double* out3, cudaStream_t s) {
    if (ntiles < 1 || ntiles > DT_NOALLOC_MAX_BLOCKS) return 1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= DT_NOALLOC_MAX_DEVICES) return 2;
    double* partial = nullptr;
    {
        // Host code cannot use the array's name as a device address: look the
        // address up once per device, with that device current.
        std::lock_guard<std::mutex> lock(g_dt_partial_mutex);
        if (!g_dt_partial_addr[dev]) {
            void* a = nullptr;
            if (cudaGetSymbolAddress(&a, g_dt_partial) != cudaSuccess) return 2;
            g_dt_partial_addr[dev] = static_cast<double*>(a);
        }
        partial = g_dt_partial_addr[dev];
    }
    // every block writes its pair before k_dt_final reads it, in stream order,
    // so nothing has to be cleared between calls
    DGFV_DISPATCH(nk, (k_dt<NK><<<ntiles, 256, 0, s>>>(P, T, U, partial)));
    k_dt_final<<<1, 1024, 0, s>>>(partial, ntiles, P.ph.viscous, cfl_c, cfl_v, out3);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

void launch_indicator(int nk, const Params& P, const double* U, int n_elem, double* Ip, double* Ih, uint8_t* dec,
                      const double thr[4], int N_min, int N_max, int vars, cudaStream_t s) {
    const Thresholds t{thr[0], thr[1], thr[2], thr[3]};
    const int nmax = std::max(N_max + 1, P.nfv), p3 = nmax * nmax * nmax;
    const size_t sm = sizeof(double) * (size_t)p3 * (nk + 4 + 2 + 2 * (nk + 1));
    DGFV_DISPATCH(nk, (cudaFuncSetAttribute(k_indicator<NK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                       k_indicator<NK><<<n_elem, 128, sm, s>>>(P, U, n_elem, Ip, Ih, dec, t, N_min, N_max, vars,
                                                                p3)));
}

void launch_remap(const Params& P, const uint8_t* n_old, const uint8_t* N_old, const uint8_t* fv_old,
                  const int64_t* off_old, const uint8_t* n_new, const uint8_t* N_new, const uint8_t* fv_new,
                  const int64_t* off_new, int V, int n_elem, const double* Uo, double* Un, int nmax,
                  cudaStream_t s) {
    RemapSide A{n_old, N_old, fv_old, off_old}, Bn{n_new, N_new, fv_new, off_new};
    const size_t sm = sizeof(double) * (size_t)(2 * V * nmax * nmax * nmax);  // t1 and t2 of the largest element
    cudaFuncSetAttribute(k_remap, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_remap<<<n_elem, 128, sm, s>>>(P, A, Bn, V, Uo, Un);
}

double probe_dmma(int iters, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    double* sink = nullptr;
    if (cudaMalloc(&sink, 1024 * sizeof(double)) != cudaSuccess) return -1.0;
    const int blocks = sms * 4, threads = 256;
    k_probe_dmma<<<blocks, threads, 0, s>>>(16, sink);  // warm-up
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
    k_probe_dmma<<<blocks, threads, 0, s>>>(iters, sink);
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    const double flops = 2.0 * 8 * 8 * 4 * 8.0 * (double)iters * blocks * (threads / 32);
    return ms > 0 ? flops / (ms * 1e-3) : -1.0;
}

double probe_dfma(int iters, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    double* sink = nullptr;
    if (cudaMalloc(&sink, 1024 * sizeof(double)) != cudaSuccess) return -1.0;
    const int blocks = sms * 8, threads = 256;
    k_probe_dfma<<<blocks, threads, 0, s>>>(16, sink);  // warm-up
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
    k_probe_dfma<<<blocks, threads, 0, s>>>(iters, sink);
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    const double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
    return ms > 0 ? flops / (ms * 1e-3) : -1.0;
}

}  // namespace dgfv
