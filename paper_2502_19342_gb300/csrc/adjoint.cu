// Adjoint (vector-Jacobian product) of R(U) for DG elements with the local
// Lax-Friedrichs flux: U_bar = (dR/dU)^T R_bar.
//
// The forward evaluation is a chain of linear maps (face traces, BR1 lifting,
// tensor-product maps between degrees, volume and surface integrals) and two
// pointwise nonlinear functions (nodal fluxes, interface fluxes).  The adjoint
// runs the chain backwards: every linear map is applied transposed and the
// pointwise functions through their hand-written reverse mode
// (physics_adj.cuh).  It needs the forward face values u(+-1), the lifting
// values U* and the gradient traces g(+-1) of the same U (the caller runs the
// forward face, lifting and volume kernels first).
//
//   k_adj_surface    R_bar -> adjoint of the outward face fluxes        (Eq. 22 surface term)^T
//   k_adj_face_conf  face-flux adjoint, conforming faces               (Eqs. 20, 21)^T
//   k_adj_mixed_*    face-flux adjoint of faces that change representation,
//                    with the transposed maps (three passes)            (Sec. 3.2.1, 3.2.2)^T
//   k_adj_volume     volume integral^T, nodal-flux adjoint, gradient
//                    trace^T, lifting^T -> U_bar (part), U*_bar          (Eqs. 22, 23)^T
//   k_adj_lift       lifting value^T (mean on the lower degree)         (Eq. 19, Sec. 3.2.2)^T
//   k_adj_prolong    face trace^T -> U_bar (rest)
#include <cuda_runtime.h>

#include "adjoint.h"
#include "common.cuh"
#include "device_util.cuh"
#include "physics_adj.cuh"

namespace dgfv {

// k_adj_surface: F*_bar on each face slot of a DG element.  The forward adds
// rh_d * lhat^{+-}_i F*_{+-d}[p] to -R at node (i along d, p).
template <int NK>
__global__ void __launch_bounds__(256) k_adj_surface(Params P, AdjBuffers A, Tiles T, const double* __restrict__ Rb) {
    constexpr int V = NK + 4;
    const int first = T.first[blockIdx.x], count = T.count[blockIdx.x], n = T.n[blockIdx.x];
    const int n2 = n * n, n3 = n2 * n, per = 6 * V * n2;
    for (int idx = threadIdx.x; idx < count * per; idx += blockDim.x) {
        const int el = idx / per, r = idx % per, f = r / (V * n2), r2 = r % (V * n2), v = r2 / n2, p = r2 % n2;
        const int e = T.items[first + el];
        const int d = f >> 1, a = p % n, b = p / n;
        const double* lh = B(P, (f & 1) ? P.bi.lhp[n] : P.bi.lhm[n]);
        const double* src = Rb + P.t.off[e] + (int64_t)v * n3;
        double s = 0.0;
        for (int i = 0; i < n; ++i) s = fma(__ldg(lh + i), src[node_index(n, d, i, a, b)], s);
        A.fbar[(P.t.fo[e] + (int64_t)f * n2) * V + v * n2 + p] = -P.t.rh[3 * e + d] * s;
    }
}

// k_adj_face_conf: faces with equal degree on both sides, one thread per point.
template <int NK, int D>
__device__ __forceinline__ void adj_conf_body(const Params& P, const AdjBuffers& A, const Faces& Fc,
                                              const int32_t* __restrict__ items, int first, int count, int nc) {
    constexpr int V = NK + 4;
    const int nc2 = nc * nc;
    for (int t = threadIdx.x; t < count * nc2; t += blockDim.x) {
        const int fid = items[first + t / nc2], p = t % nc2;
        const int eL = Fc.L[fid], eR = Fc.R[fid];
        const int64_t sL = P.t.fo[eL] + (int64_t)(2 * D + 1) * nc2;
        const int64_t sR = P.t.fo[eR] + (int64_t)(2 * D) * nc2;
        double uL[V], uR[V], gL[3 * V], gR[3 * V], Fb[V];
        double uLb[V] = {}, uRb[V] = {}, gLb[3 * V] = {}, gRb[3 * V] = {};
        const bool fv = P.t.fv[eL];  // conforming faces: both sides FV or both DG
        const double* us = fv ? P.b.frec : P.b.fu;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            uL[v] = us[sL * V + v * nc2 + p];
            uR[v] = us[sR * V + v * nc2 + p];
            // L's slot holds +F, R's slot -F
            Fb[v] = A.fbar[sL * V + v * nc2 + p] - A.fbar[sR * V + v * nc2 + p];
        }
        // both gradient traces loaded up front (their latency overlaps the
        // convective reverse; measured faster here than reading each side
        // just before its viscous reverse)
        if (P.ph.viscous) {
#pragma unroll
            for (int x = 0; x < 3 * V; ++x) {
                gL[x] = P.b.fg[sL * 3 * V + x * nc2 + p];
                gR[x] = P.b.fg[sR * 3 * V + x * nc2 + p];
            }
        }
        face_point_rev<NK, D>(P.ph, uL, gL, uR, gR, D, Fb, uLb, gLb, uRb, gRb, fv);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            A.ubar[sL * V + v * nc2 + p] = uLb[v];
            A.ubar[sR * V + v * nc2 + p] = uRb[v];
        }
#pragma unroll
        for (int x = 0; x < 3 * V; ++x) {
            A.gbar[sL * 3 * V + x * nc2 + p] = gLb[x];
            A.gbar[sR * 3 * V + x * nc2 + p] = gRb[x];
        }
    }
}

template <int NK>
__global__ void __launch_bounds__(128) k_adj_face_conf(Params P, AdjBuffers A, Faces Fc, FaceTiles T) {
    const int first = T.first[blockIdx.x], count = T.count[blockIdx.x], nc = T.nc[blockIdx.x];
    switch (T.d[blockIdx.x]) {
        case 0: adj_conf_body<NK, 0>(P, A, Fc, T.items, first, count, nc); break;
        case 1: adj_conf_body<NK, 1>(P, A, Fc, T.items, first, count, nc); break;
        default: adj_conf_body<NK, 2>(P, A, Fc, T.items, first, count, nc); break;
    }
}

// Mixed faces in three passes, like the forward (and on its tiles and scratch):
// k_adj_mixed_in (one CTA per face): the mapped side's forward u, g on the
// common representation into Sin (4V per point), and the flux adjoint there,
// F_bar = sgn_direct fbar_direct + sgn_mapped M_out^T fbar_mapped, into Sout;
// k_adj_mixed_point (one thread per common point): the point-flux reverse, the
// direct side's ubar/gbar written in place, the mapped side's into Sin;
// k_adj_mixed_out (one CTA per face): M_in^T back onto the mapped side's slots.
// M_in / M_out: V^{N->Nc} / its L2 projection back, or V^{DG->FV} / V^{FV->DG}.
template <int NK>
__global__ void __launch_bounds__(128) k_adj_mixed_in(Params P, AdjBuffers A, Faces Fc, const int32_t* __restrict__ mface,
                                                      const int64_t* __restrict__ mpt, double* __restrict__ Sin,
                                                      double* __restrict__ Sout) {
    constexpr int V = NK + 4;
    __shared__ double tmp[3 * V * MAXP * MAXP], sb[V * MAXP * MAXP];
    const int k = blockIdx.x, fid = mface[k], d = Fc.d[fid];
    const MixedFace m = mixed_face(P, Fc, fid);
    const int em = m.mapL ? m.eL : m.eR, fm = m.mapL ? 2 * d + 1 : 2 * d, n = P.t.n[em], n2 = n * n;
    const int ed = m.mapL ? m.eR : m.eL, fd = m.mapL ? 2 * d : 2 * d + 1, nc2 = m.nc * m.nc;
    const int64_t slot = P.t.fo[em] + (int64_t)fm * n2, sd = P.t.fo[ed] + (int64_t)fd * nc2;
    // a coarser FV side (per-element counts) enters by its sub-cell overlaps,
    // from its reconstructed face states, as in k_mixed_in / k_mixed_out
    const bool fvs = P.t.fv[em];
    const double* Min = B(P, fvs ? P.bi.ov[n][m.nc] : (m.cfv ? P.bi.d2f[n][m.nc] : P.bi.vm[n][m.nc]));
    const double* Mout = B(P, fvs ? P.bi.ov[m.nc][n] : (m.cfv ? P.bi.f2d[n][m.nc] : P.bi.vm[m.nc][n]));
    double* in = Sin + mpt[k] * 4 * V;
    face_map((fvs ? P.b.frec : P.b.fu) + slot * V, n, in, m.nc, Min, V, tmp);
    if (P.ph.viscous) face_map(P.b.fg + slot * 3 * V, n, in + V * nc2, m.nc, Min, 3 * V, tmp);
    // L's slot holds +F, R's slot -F
    const double sm = m.mapL ? 1.0 : -1.0;
    face_map_t(A.fbar + slot * V, n, sb, m.nc, Mout, V, tmp);
    double* out = Sout + mpt[k] * V;
    for (int i = threadIdx.x; i < V * nc2; i += blockDim.x) out[i] = sm * sb[i] - sm * A.fbar[sd * V + i];
}

template <int NK, int D>
__device__ __forceinline__ void adj_mixed_point_body(const Params& P, const AdjBuffers& A, const Faces& Fc,
                                                     const int32_t* __restrict__ mface, const int64_t* __restrict__ mpt,
                                                     double* __restrict__ Sin, const double* __restrict__ Sout,
                                                     const int32_t* __restrict__ items, int first, int count, int nc) {
    constexpr int V = NK + 4;
    const int nc2 = nc * nc;
    for (int t = threadIdx.x; t < count * nc2; t += blockDim.x) {
        const int k = items[first + t / nc2], p = t % nc2;
        const MixedFace m = mixed_face(P, Fc, mface[k]);
        const int ed = m.mapL ? m.eR : m.eL, fd = m.mapL ? 2 * D : 2 * D + 1;
        const int64_t sd = P.t.fo[ed] + (int64_t)fd * nc2;
        const double* ud = (P.t.fv[ed] ? P.b.frec : P.b.fu) + sd * V + p;
        const double* gd = P.b.fg + sd * 3 * V + p;
        double* um = Sin + mpt[k] * 4 * V + p;
        double* gm = um + V * nc2;
        const double* fb = Sout + mpt[k] * V + p;
        double uL[V], uR[V], Fb[V];
        double uLb[V] = {}, uRb[V] = {};
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const double a = um[v * nc2], b = ud[v * nc2];
            uL[v] = m.mapL ? a : b;
            uR[v] = m.mapL ? b : a;
            Fb[v] = fb[v * nc2];
        }
        double* gbd = A.gbar + sd * 3 * V + p;
        // viscous sides one after the other; the mapped side's gradient adjoint
        // replaces its gradient in Sin once that side is done
        face_point_rev_seq<NK, D>(
            P.ph, uL, uR, D, Fb, uLb, uRb, m.cfv,
            [&](int side, double* g) {
                const double* src = (side == 0) == m.mapL ? gm : gd;
#pragma unroll
                for (int x = 0; x < 3 * V; ++x) g[x] = src[x * nc2];
            },
            [&](int side, const double* gb) {
                double* dst = (side == 0) == m.mapL ? gm : gbd;
#pragma unroll
                for (int x = 0; x < 3 * V; ++x) dst[x * nc2] = gb[x];
            });
        double* ubd = A.ubar + sd * V + p;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            ubd[v * nc2] = m.mapL ? uRb[v] : uLb[v];
            um[v * nc2] = m.mapL ? uLb[v] : uRb[v];
        }
    }
}

template <int NK>
__global__ void __launch_bounds__(128) k_adj_mixed_point(Params P, AdjBuffers A, Faces Fc, FaceTiles T,
                                                         const int32_t* __restrict__ mface,
                                                         const int64_t* __restrict__ mpt, double* __restrict__ Sin,
                                                         const double* __restrict__ Sout) {
    const int first = T.first[blockIdx.x], count = T.count[blockIdx.x], nc = T.nc[blockIdx.x];
    switch (T.d[blockIdx.x]) {
        case 0: adj_mixed_point_body<NK, 0>(P, A, Fc, mface, mpt, Sin, Sout, T.items, first, count, nc); break;
        case 1: adj_mixed_point_body<NK, 1>(P, A, Fc, mface, mpt, Sin, Sout, T.items, first, count, nc); break;
        default: adj_mixed_point_body<NK, 2>(P, A, Fc, mface, mpt, Sin, Sout, T.items, first, count, nc); break;
    }
}

template <int NK>
__global__ void __launch_bounds__(128) k_adj_mixed_out(Params P, AdjBuffers A, Faces Fc, const int32_t* __restrict__ mface,
                                                       const int64_t* __restrict__ mpt, const double* __restrict__ Sin) {
    constexpr int V = NK + 4;
    __shared__ double tmp[3 * V * MAXP * MAXP];
    const int k = blockIdx.x, fid = mface[k], d = Fc.d[fid];
    const MixedFace m = mixed_face(P, Fc, fid);
    const int em = m.mapL ? m.eL : m.eR, fm = m.mapL ? 2 * d + 1 : 2 * d, n = P.t.n[em], n2 = n * n;
    const int64_t slot = P.t.fo[em] + (int64_t)fm * n2;
    const double* Min =
        B(P, P.t.fv[em] ? P.bi.ov[n][m.nc] : (m.cfv ? P.bi.d2f[n][m.nc] : P.bi.vm[n][m.nc]));
    const double* in = Sin + mpt[k] * 4 * V;
    face_map_t(in, m.nc, A.ubar + slot * V, n, Min, V, tmp);
    if (P.ph.viscous) face_map_t(in + V * m.nc * m.nc, m.nc, A.gbar + slot * 3 * V, n, Min, 3 * V, tmp);
}

// Volume adjoint in three kernels around the face adjoint.
// k_adj_vol_a: per tile of DG elements (shared memory 3V n^3 doubles per element):
//   g (lifted gradient) recomputed from U and U*, its face traces written for
//   the face adjoint; g and F_bar_d = -rh_d Dhat^T R_bar (volume integral^T)
//   written per node (6V values) for k_adj_point.
template <int NK, int NP>
__device__ __forceinline__ void adj_vol_a_body(const Params& P, const Tiles& T, const double* __restrict__ U,
                                               const double* __restrict__ Rb, double* __restrict__ gf) {
    constexpr int V = NK + 4;
    extern __shared__ double sm[];
    const int first = T.first[blockIdx.x], count = T.count[blockIdx.x];
    const int n = NP > 0 ? NP : T.n[blockIdx.x];
    const int n2 = n * n, n3 = n2 * n;
    double* sD = sm;
    double* sl = sD + n * n;               // lm, lp, lhm, lhp
    double* sG = sl + 4 * n;               // count * 3V n^3: g
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) sD[i] = B(P, P.bi.dhat[n])[i];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        sl[i] = B(P, P.bi.lm[n])[i];
        sl[n + i] = B(P, P.bi.lp[n])[i];
        sl[2 * n + i] = B(P, P.bi.lhm[n])[i];
        sl[3 * n + i] = B(P, P.bi.lhp[n])[i];
    }
    __syncthreads();
    const bool visc = P.ph.viscous;
    const int per = 3 * V * n3;
    for (int idx = threadIdx.x; idx < count * per; idx += blockDim.x) {
        const int el = idx / per, r = idx % per, d = r / (V * n3), r2 = r % (V * n3), v = r2 / n3, c = r2 % n3;
        const int e = T.items[first + el];
        const int i = c % n, j = (c / n) % n, k = c / n2;
        const int m0 = d == 0 ? i : (d == 1 ? j : k);
        const int a = d == 0 ? j : i, b = d == 2 ? j : k;
        const int p = a + n * b;
        const double rh = P.t.rh[3 * e + d];
        double* out = gf + 6 * P.t.off[e];  // [g (3V x n3) | F_bar (3V x n3)] per element
        const double* rsrc = Rb + P.t.off[e] + (int64_t)v * n3;
        double fb = 0.0;
        for (int q = 0; q < n; ++q) fb = fma(sD[q * n + m0], rsrc[node_index(n, d, q, a, b)], fb);
        out[per + r] = -rh * fb;
        if (visc) {
            const double* src = U + P.t.off[e] + (int64_t)v * n3;
            const int64_t fo = P.t.fo[e];
            double s = 0.0;
            for (int m = 0; m < n; ++m) s = fma(sD[m0 * n + m], src[node_index(n, d, m, a, b)], s);
            s = fma(sl[3 * n + m0], P.b.flift[(fo + (int64_t)(2 * d + 1) * n2) * V + v * n2 + p], s);
            s = fma(-sl[2 * n + m0], P.b.flift[(fo + (int64_t)(2 * d) * n2) * V + v * n2 + p], s);
            sG[el * per + r] = rh * s;
            out[r] = rh * s;
        }
    }
    if (!visc) return;
    __syncthreads();
    // gradient traces for the face adjoint
    const int pt = 6 * 3 * V * n2;
    for (int idx = threadIdx.x; idx < count * pt; idx += blockDim.x) {
        const int el = idx / pt, r = idx % pt, f = r / (3 * V * n2), r2 = r % (3 * V * n2), x = r2 / n2, p = r2 % n2;
        const int e = T.items[first + el];
        const int d = f >> 1, a = p % n, b = p / n;
        const double* lb = sl + ((f & 1) ? n : 0);
        const double* src = sG + el * per + x * n3;
        double s = 0.0;
        for (int m = 0; m < n; ++m) s = fma(lb[m], src[node_index(n, d, m, a, b)], s);
        P.b.fg[(P.t.fo[e] + (int64_t)f * n2) * 3 * V + x * n2 + p] = s;
    }
}

template <int NK>
__global__ void __launch_bounds__(256) k_adj_vol_a(Params P, Tiles T, const double* __restrict__ U,
                                                   const double* __restrict__ Rb, double* __restrict__ gf) {
    switch (T.n[blockIdx.x]) {  // the tile's point count as a compile-time constant
        case 2: adj_vol_a_body<NK, 2>(P, T, U, Rb, gf); break;
        case 3: adj_vol_a_body<NK, 3>(P, T, U, Rb, gf); break;
        case 4: adj_vol_a_body<NK, 4>(P, T, U, Rb, gf); break;
        case 5: adj_vol_a_body<NK, 5>(P, T, U, Rb, gf); break;
        case 6: adj_vol_a_body<NK, 6>(P, T, U, Rb, gf); break;
        case 7: adj_vol_a_body<NK, 7>(P, T, U, Rb, gf); break;
        default: adj_vol_a_body<NK, 8>(P, T, U, Rb, gf); break;
    }
}

// k_adj_point: nodal-flux reverse, one thread per DG node (no shared memory, no
// barriers): U_bar (direct part) and g_bar (to gvol) from u, g and F_bar.
template <int NK>
__global__ void __launch_bounds__(128) k_adj_point(Params P, Tiles T, const double* __restrict__ U,
                                                   const double* __restrict__ gf, double* __restrict__ Ub,
                                                   double* __restrict__ gvol, int split) {
    constexpr int V = NK + 4;
    const int first = T.first[blockIdx.x], count = T.count[blockIdx.x], n = T.n[blockIdx.x];
    const int n3 = n * n * n, per = 3 * V * n3;
    const bool visc = P.ph.viscous;
    for (int idx = threadIdx.x; idx < count * n3; idx += blockDim.x) {
        const int el = idx / n3, c = idx % n3;
        const int e = T.items[first + el];
        const int64_t off = P.t.off[e];
        const double* in = gf + 6 * off + c;
        double u[V], g[3 * V], Fb[3 * V], ub[V] = {}, gb[3 * V] = {};
#pragma unroll
        for (int v = 0; v < V; ++v) u[v] = U[off + (int64_t)v * n3 + c];
#pragma unroll
        for (int x = 0; x < 3 * V; ++x) {
            Fb[x] = in[(per + x * n3)];
            g[x] = visc ? in[x * n3] : 0.0;
        }
        volume_point_rev<NK>(P.ph, u, g, Fb, ub, gb, !split);  // split form: k_adj_split has the convective part
#pragma unroll
        for (int v = 0; v < V; ++v) Ub[off + (int64_t)v * n3 + c] = ub[v];
        if (visc)
#pragma unroll
            for (int x = 0; x < 3 * V; ++x) gvol[3 * off + (int64_t)x * n3 + c] = gb[x];
    }
}

// k_adj_split (split form on LGL nodes, Sec. 3.5): reverse of the two-point
// volume term -rh_d sum_m S_im F#(t_i, t_m) of R_i.  Per tile: the tuples of
// every node; one thread per line (element, direction d, (a, b)) visits every
// pair i <= m once, F#_bar = -rh_d (S_im R_bar_i + S_mi R_bar_m) (the diagonal
// -rh_d S_ii R_bar_i), and adds the tuple adjoints of both nodes (shared-memory
// atomics: the three directions meet at every node); per node the tuple and
// primitive reverses add to U_bar.
template <int NK, int NP>
__device__ __forceinline__ void adj_split_body(const Params& P, const Tiles& T, const double* __restrict__ U,
                                               const double* __restrict__ Rb, double* __restrict__ Ub) {
    constexpr int V = NK + 4, NT = 6 + NK;
    extern __shared__ double sm[];
    const int first = T.first[blockIdx.x], count = T.count[blockIdx.x];
    const int n = NP > 0 ? NP : T.n[blockIdx.x];
    const int n2 = n * n, n3 = n2 * n;
    double* sS = sm;                    // n*n split matrix
    double* sK = sS + n * n;            // count * NT * n3 tuples
    double* sKb = sK + count * NT * n3; // count * NT * n3 tuple adjoints
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) sS[i] = B(P, P.bi.dsplit[n])[i];
    for (int idx = threadIdx.x; idx < count * n3; idx += blockDim.x) {
        const int el = idx / n3, c = idx % n3;
        const double* src = U + P.t.off[T.items[first + el]] + c;
        double u[V], t[NT];
#pragma unroll
        for (int v = 0; v < V; ++v) u[v] = src[(int64_t)v * n3];
        Prim<NK> s;
        prim<NK>(P.ph, u, s);
        kep_tuple<NK>(s, t);
#pragma unroll
        for (int q = 0; q < NT; ++q) {
            sK[(el * NT + q) * n3 + c] = t[q];
            sKb[(el * NT + q) * n3 + c] = 0.0;
        }
    }
    __syncthreads();
    const int lines = 3 * n2;
    for (int idx = threadIdx.x; idx < count * lines; idx += blockDim.x) {
        const int el = idx / lines, r = idx % lines, d = r / n2, p = r % n2, a = p % n, b = p / n;
        const int e = T.items[first + el];
        const double rh = P.t.rh[3 * e + d];
        const double* K = sK + el * NT * n3;
        double* Kb = sKb + el * NT * n3;
        const double* R = Rb + P.t.off[e];
        for (int i = 0; i < n; ++i) {
            const int ci = node_index(n, d, i, a, b);
            double ti[NT], Ri[V];
#pragma unroll
            for (int q = 0; q < NT; ++q) ti[q] = K[q * n3 + ci];
#pragma unroll
            for (int v = 0; v < V; ++v) Ri[v] = R[(int64_t)v * n3 + ci];
            for (int m = i; m < n; ++m) {
                const int cm = node_index(n, d, m, a, b);
                double tm[NT], Fb[V], tb[NT];
#pragma unroll
                for (int q = 0; q < NT; ++q) {
                    tm[q] = K[q * n3 + cm];
                    tb[q] = 0.0;
                }
                const double Sim = sS[i * n + m], Smi = sS[m * n + i];
#pragma unroll
                for (int v = 0; v < V; ++v)
                    Fb[v] = -rh * (m == i ? Sim * Ri[v] : fma(Sim, Ri[v], Smi * R[(int64_t)v * n3 + cm]));
                kep_flux_rev<NK>(ti, tm, d, Fb, tb);
#pragma unroll
                for (int q = 0; q < NT; ++q) {
                    atomicAdd(&Kb[q * n3 + ci], tb[q]);
                    atomicAdd(&Kb[q * n3 + cm], tb[q]);
                }
            }
        }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < count * n3; idx += blockDim.x) {
        const int el = idx / n3, c = idx % n3;
        const int64_t off = P.t.off[T.items[first + el]];
        double u[V], tb[NT], ub[V] = {};
#pragma unroll
        for (int v = 0; v < V; ++v) u[v] = U[off + (int64_t)v * n3 + c];
#pragma unroll
        for (int q = 0; q < NT; ++q) tb[q] = sKb[(el * NT + q) * n3 + c];
        Prim<NK> s;
        prim<NK>(P.ph, u, s);
        PrimBar<NK> bb;
        zero(bb);
        kep_tuple_rev<NK>(s, tb, bb);
        prim_rev<NK>(P.ph, u, s, bb, ub);
#pragma unroll
        for (int v = 0; v < V; ++v) Ub[off + (int64_t)v * n3 + c] += ub[v];
    }
}

template <int NK>
__global__ void __launch_bounds__(256) k_adj_split(Params P, Tiles T, const double* __restrict__ U,
                                                   const double* __restrict__ Rb, double* __restrict__ Ub) {
    adj_split_body<NK, 0>(P, T, U, Rb, Ub);
}

// k_adj_vol_b (viscous only): g_bar += trace^T of the face gradient adjoints;
// lifting^T: U_bar += rh_d Dhat^T g_bar^d and U*_bar = +-rh_d lhat^{+-}^T g_bar^d.
template <int NK, int NP>
__device__ __forceinline__ void adj_vol_b_body(const Params& P, const AdjBuffers& A, const Tiles& T,
                                               const double* __restrict__ gvol, double* __restrict__ Ub) {
    constexpr int V = NK + 4;
    extern __shared__ double sm[];
    const int first = T.first[blockIdx.x], count = T.count[blockIdx.x];
    const int n = NP > 0 ? NP : T.n[blockIdx.x];
    const int n2 = n * n, n3 = n2 * n;
    double* sD = sm;
    double* sl = sD + n * n;
    double* sG = sl + 4 * n;  // count * 3V n^3: g_bar
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) sD[i] = B(P, P.bi.dhat[n])[i];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        sl[i] = B(P, P.bi.lm[n])[i];
        sl[n + i] = B(P, P.bi.lp[n])[i];
        sl[2 * n + i] = B(P, P.bi.lhm[n])[i];
        sl[3 * n + i] = B(P, P.bi.lhp[n])[i];
    }
    __syncthreads();
    const int per = 3 * V * n3;
    for (int idx = threadIdx.x; idx < count * per; idx += blockDim.x) {
        const int el = idx / per, r = idx % per, x = r / n3, c = r % n3;
        const int e = T.items[first + el];
        const int ijk[3] = {c % n, (c / n) % n, c / n2};
        const int64_t fo = P.t.fo[e];
        double acc = gvol[3 * P.t.off[e] + r];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int m0 = ijk[d];
            const int p = (d == 0 ? ijk[1] : ijk[0]) + n * (d == 2 ? ijk[1] : ijk[2]);
            acc = fma(sl[m0], A.gbar[(fo + (int64_t)(2 * d) * n2) * 3 * V + x * n2 + p], acc);
            acc = fma(sl[n + m0], A.gbar[(fo + (int64_t)(2 * d + 1) * n2) * 3 * V + x * n2 + p], acc);
        }
        sG[el * per + r] = acc;
    }
    __syncthreads();
    const int pv = V * n3;
    for (int idx = threadIdx.x; idx < count * pv; idx += blockDim.x) {
        const int el = idx / pv, r = idx % pv, v = r / n3, c = r % n3;
        const int e = T.items[first + el];
        const int ijk[3] = {c % n, (c / n) % n, c / n2};
        double acc = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int m0 = ijk[d];
            const int a = d == 0 ? ijk[1] : ijk[0], b = d == 2 ? ijk[1] : ijk[2];
            const double* gsrc = sG + el * per + (d * V + v) * n3;
            double s = 0.0;
            for (int i = 0; i < n; ++i) s = fma(sD[i * n + m0], gsrc[node_index(n, d, i, a, b)], s);
            acc = fma(P.t.rh[3 * e + d], s, acc);
        }
        Ub[P.t.off[e] + r] += acc;
    }
    const int pf = 6 * V * n2;
    for (int idx = threadIdx.x; idx < count * pf; idx += blockDim.x) {
        const int el = idx / pf, r = idx % pf, f = r / (V * n2), r2 = r % (V * n2), v = r2 / n2, p = r2 % n2;
        const int e = T.items[first + el];
        const int d = f >> 1, a = p % n, b = p / n;
        const double* lh = sl + ((f & 1) ? 3 * n : 2 * n);
        const double* gsrc = sG + el * per + (d * V + v) * n3;
        double s = 0.0;
        for (int i = 0; i < n; ++i) s = fma(lh[i], gsrc[node_index(n, d, i, a, b)], s);
        A.sbar[(P.t.fo[e] + (int64_t)f * n2) * V + v * n2 + p] = ((f & 1) ? 1.0 : -1.0) * P.t.rh[3 * e + d] * s;
    }
}

template <int NK>
__global__ void __launch_bounds__(256) k_adj_vol_b(Params P, AdjBuffers A, Tiles T, const double* __restrict__ gvol,
                                                   double* __restrict__ Ub) {
    switch (T.n[blockIdx.x]) {  // the tile's point count as a compile-time constant
        case 2: adj_vol_b_body<NK, 2>(P, A, T, gvol, Ub); break;
        case 3: adj_vol_b_body<NK, 3>(P, A, T, gvol, Ub); break;
        case 4: adj_vol_b_body<NK, 4>(P, A, T, gvol, Ub); break;
        case 5: adj_vol_b_body<NK, 5>(P, A, T, gvol, Ub); break;
        case 6: adj_vol_b_body<NK, 6>(P, A, T, gvol, Ub); break;
        case 7: adj_vol_b_body<NK, 7>(P, A, T, gvol, Ub); break;
        default: adj_vol_b_body<NK, 8>(P, A, T, gvol, Ub); break;
    }
}

// k_adj_lift: lifting value^T per face (both sides DG).  Forward on the lower
// degree m: avg = (P_{nL->m} uL + P_{nR->m} uR)/2, U*_side = I_{m->n_side} avg.
template <int NK>
__global__ void __launch_bounds__(64) k_adj_lift(Params P, AdjBuffers A, Faces Fc, const int32_t* __restrict__ list) {
    constexpr int V = NK + 4, PP = MAXP * MAXP;
    __shared__ double sA[V * PP], sB[V * PP], sT[V * PP];
    const int fid = list[blockIdx.x];
    const int eL = Fc.L[fid], eR = Fc.R[fid], d = Fc.d[fid];
    const bool fvL = P.t.fv[eL], fvR = P.t.fv[eR];
    if (fvL && fvR) return;
    const int nL = P.t.n[eL], nR = P.t.n[eR];
    const int64_t sL = (P.t.fo[eL] + (int64_t)(2 * d + 1) * nL * nL) * V;
    const int64_t sR = (P.t.fo[eR] + (int64_t)(2 * d) * nR * nR) * V;
    if (fvL || fvR) {
        // U*_DG = (u_DG + V^{FV->DG} rec_FV)/2: u_DG_bar += U*_bar/2, and the FV
        // reconstructed face state's adjoint += V^{FV->DG}^T U*_bar/2
        const int nD = fvL ? nR : nL, nF = fvL ? nL : nR;  // the FV side's own count
        const int64_t sD = fvL ? sR : sL, sF = fvL ? sL : sR;
        for (int i = threadIdx.x; i < V * nD * nD; i += blockDim.x) {
            const double a = 0.5 * A.sbar[sD + i];
            A.ubar[sD + i] += a;
            sA[i] = a;
        }
        __syncthreads();
        face_map_t(sA, nD, sB, nF, B(P, P.bi.f2d[nD][nF]), V, sT);
        for (int i = threadIdx.x; i < V * nF * nF; i += blockDim.x) A.ubar[sF + i] += sB[i];
        return;
    }
    if (nL == nR) {
        for (int i = threadIdx.x; i < V * nL * nL; i += blockDim.x) {
            const double a = 0.5 * (A.sbar[sL + i] + A.sbar[sR + i]);
            A.ubar[sL + i] += a;
            A.ubar[sR + i] += a;
        }
        return;
    }
    const bool lowL = nL < nR;
    const int m = lowL ? nL : nR, M = lowL ? nR : nL;
    const int64_t sLo = lowL ? sL : sR, sHi = lowL ? sR : sL;
    // avg_bar = U*_bar_lo + I^T U*_bar_hi
    for (int i = threadIdx.x; i < V * M * M; i += blockDim.x) sA[i] = A.sbar[sHi + i];
    __syncthreads();
    face_map_t(sA, M, sB, m, B(P, P.bi.vm[m][M]), V, sT);
    for (int i = threadIdx.x; i < V * m * m; i += blockDim.x) {
        const double a = 0.5 * (sB[i] + A.sbar[sLo + i]);
        A.ubar[sLo + i] += a;
        sB[i] = a;
    }
    __syncthreads();
    face_map_t(sB, m, sA, M, B(P, P.bi.vm[M][m]), V, sT);  // projection^T
    for (int i = threadIdx.x; i < V * M * M; i += blockDim.x) A.ubar[sHi + i] += sA[i];
}

// ---------------------------------------------------------------------------------
// FV sub-cell elements (Sec. 3.1.2), reversed.
//
// k_adj_surface_fv: the forward adds (n/h_d) F*_f at the boundary sub-cells to
// -R, so F*_f_bar = -(n/h_d) R_bar there.
template <int NK>
__global__ void __launch_bounds__(128) k_adj_surface_fv(Params P, AdjBuffers A, Tiles T, const double* __restrict__ Rb) {
    constexpr int V = NK + 4;
    const int e = T.items[T.first[blockIdx.x]], n = P.t.n[e], n2 = n * n, n3 = n2 * n;
    for (int i = threadIdx.x; i < 6 * V * n2; i += blockDim.x) {
        const int f = i / (V * n2), r = i % (V * n2), v = r / n2, p = r % n2, d = f >> 1;
        const int c = node_index(n, d, (f & 1) ? n - 1 : 0, p % n, p / n);
        A.fbar[(P.t.fo[e] + (int64_t)f * n2) * V + v * n2 + p] =
            -0.5 * n * P.t.rh[3 * e + d] * Rb[P.t.off[e] + (int64_t)v * n3 + c];
    }
}

// k_adj_prolong: U_bar += trace^T of the face-value adjoints.
template <int NK>
__global__ void __launch_bounds__(256) k_adj_prolong(Params P, AdjBuffers A, Tiles T, double* __restrict__ Ub) {
    constexpr int V = NK + 4;
    const int first = T.first[blockIdx.x], count = T.count[blockIdx.x], n = T.n[blockIdx.x];
    const int n2 = n * n, n3 = n2 * n, per = V * n3;
    const double* lm = B(P, P.bi.lm[n]);
    const double* lp = B(P, P.bi.lp[n]);
    for (int idx = threadIdx.x; idx < count * per; idx += blockDim.x) {
        const int el = idx / per, r = idx % per, v = r / n3, c = r % n3;
        const int e = T.items[first + el];
        const int ijk[3] = {c % n, (c / n) % n, c / n2};
        const int64_t fo = P.t.fo[e];
        double acc = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int m0 = ijk[d];
            const int p = (d == 0 ? ijk[1] : ijk[0]) + n * (d == 2 ? ijk[1] : ijk[2]);
            acc = fma(__ldg(lm + m0), A.ubar[(fo + (int64_t)(2 * d) * n2) * V + v * n2 + p], acc);
            acc = fma(__ldg(lp + m0), A.ubar[(fo + (int64_t)(2 * d + 1) * n2) * V + v * n2 + p], acc);
        }
        Ub[P.t.off[e] + r] += acc;
    }
}

// out = a*x + b*y (element-wise over n doubles)
__global__ void k_axpby(int64_t n, double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                        double* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = fma(a, x[i], b * y[i]);
}

// The stage combinations of the SSP-RK3 step adjoint, one pass each:
//   mode 0: o1 = c1 (x + dt y), o2 = c2 x          (after the VJP at U2)
//   mode 1: o1 = c1 (x + dt y), o2 += c2 x         (after the VJP at U1)
//   mode 2: o2 += x + dt y                         (after the VJP at U0)
__global__ void k_rk3_adj_combine(int64_t n, int mode, double c1, double c2, double dt, const double* __restrict__ x,
                                  const double* __restrict__ y, double* __restrict__ o1, double* __restrict__ o2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double xi = x[i], t = fma(dt, y[i], xi);
        if (mode == 0) {
            o1[i] = c1 * t;
            o2[i] = c2 * xi;
        } else if (mode == 1) {
            o1[i] = c1 * t;
            o2[i] = fma(c2, xi, o2[i]);
        } else {
            o2[i] += t;
        }
    }
}

// ================================================================= launchers
// ---------------------------------------------------------------------------------
// Mortars (Sec. 3.2.3), transposed.  The forward projects the virtual small
// sides' fluxes and lifting values onto the big side, F_0 = sum_q P_q F_q, and
// interpolates the big side's traces to them, u_q = M_q u_0, g_q = M_q g_0
// (P_q, M_q tensor products of the per-direction maps; DG big sides only, the
// adjoint has no FV elements).
//   k_adj_mortar_virt: which 0: fbar_q = P_q^T fbar_0, which 1: sbar_q = P_q^T sbar_0
//                      (one CTA per virtual side)
//   k_adj_mortar_big:  which 0: gbar_0 = sum_q M_q^T gbar_q, which 1: ubar_0 = sum_q M_q^T ubar_q
//                      (one CTA per mortar; no face writes the big side's slot)
__device__ __forceinline__ const double* adj_mortar_dir(const Params& P, int split, int quad, int dir, int n,
                                                        bool proj, bool fv = false) {
    if (!((split >> dir) & 1)) return B(P, P.bi.eye[n]);
    const int h = (quad >> dir) & 1;
    if (fv) return B(P, proj ? P.bi.mfp[h] : P.bi.mfi[h]);
    return B(P, proj ? P.bi.mp[n][h] : P.bi.mi[n][h]);
}

template <int NK>
__global__ void __launch_bounds__(128) k_adj_mortar_virt(Params P, AdjBuffers A, MortarTables M, int which) {
    constexpr int V = NK + 4;
    __shared__ double tmp[V * MAXP * MAXP];
    const int v = M.n_elem + blockIdx.x, m = M.vmort[blockIdx.x], q = M.vquad[blockIdx.x];
    const int eb = M.big[m], fB = M.fB[m], sp = M.split[m], n = P.t.n[eb], n2 = n * n;
    const bool fv = P.t.fv[eb];
    if (which == 1 && fv) return;  // an FV big side has no lifting value
    double* buf = which == 0 ? A.fbar : A.sbar;
    face_map2_t(buf + (P.t.fo[eb] + (int64_t)fB * n2) * V, n, buf + (P.t.fo[v] + (int64_t)fB * n2) * V, n,
                adj_mortar_dir(P, sp, q, 0, n, true, fv), adj_mortar_dir(P, sp, q, 1, n, true, fv), V, tmp);
}

template <int NK>
__global__ void __launch_bounds__(128) k_adj_mortar_big(Params P, AdjBuffers A, MortarTables M, int which) {
    constexpr int V = NK + 4;
    __shared__ double tmp[3 * V * MAXP * MAXP], res[3 * V * MAXP * MAXP], acc[3 * V * MAXP * MAXP];
    const int m = blockIdx.x, eb = M.big[m], fB = M.fB[m], sp = M.split[m], n = P.t.n[eb], n2 = n * n;
    const bool fv = P.t.fv[eb];  // FV big side: the adjoints of its reconstructed state and boundary gradient
    const int w = which == 0 ? 3 * V : V;
    double* buf = which == 0 ? A.gbar : A.ubar;
    for (int i = threadIdx.x; i < w * n2; i += blockDim.x) acc[i] = 0.0;
    for (int vi = M.vfirst[m]; vi < M.vfirst[m + 1]; ++vi) {
        const int v = M.n_elem + vi, q = M.vquad[vi];
        face_map2_t(buf + (P.t.fo[v] + (int64_t)fB * n2) * w, n, res, n, adj_mortar_dir(P, sp, q, 0, n, false, fv),
                    adj_mortar_dir(P, sp, q, 1, n, false, fv), w, tmp);
        for (int i = threadIdx.x; i < w * n2; i += blockDim.x) acc[i] += res[i];
        __syncthreads();
    }
    double* dst = buf + (P.t.fo[eb] + (int64_t)fB * n2) * w;
    for (int i = threadIdx.x; i < w * n2; i += blockDim.x) dst[i] = acc[i];
}

// k_adj_mortar_nb: one CTA per mortar; the transposes of k_mortar_nb's
// neighbour values of FV elements (left by k_adj_fv, in conservative
// variables, in the owner's fbar slot of the mortar face): an FV small side
// read the big element's layer through M^FV_0q, an FV big side the small
// elements' layers through M^FV_q0.  The layer adjoints go into the elements'
// U_bar with atomics (an element can sit on two mortars).
template <int NK>
__global__ void __launch_bounds__(128) k_adj_mortar_nb(Params P, AdjBuffers A, MortarTables M, double* __restrict__ Ub) {
    constexpr int V = NK + 4, PP = MAXP * MAXP;
    __shared__ double acc[V * PP], res[V * PP], sT1[V * PP], sT2[V * PP];
    const int m = blockIdx.x, eb = M.big[m], fB = M.fB[m], fS = fB ^ 1, sp = M.split[m];
    const int n = P.nfv, n2 = n * n;
    bool any = false;
    for (int i = threadIdx.x; i < V * n2; i += blockDim.x) acc[i] = 0.0;
    for (int vi = M.vfirst[m]; vi < M.vfirst[m + 1]; ++vi) {
        const int q = M.vsmall[vi], qd = M.vquad[vi];
        if (!P.t.fv[q]) continue;
        any = true;
        face_map2_t(A.fbar + (P.t.fo[q] + (int64_t)fS * n2) * V, n, res, n, adj_mortar_dir(P, sp, qd, 0, n, false, true),
                    adj_mortar_dir(P, sp, qd, 1, n, false, true), V, sT1);
        for (int i = threadIdx.x; i < V * n2; i += blockDim.x) acc[i] += res[i];
        __syncthreads();
    }
    if (any) fv_layer_t<NK, true>(P, eb, fB, n, acc, Ub, sT1, sT2);
    if (!P.t.fv[eb]) return;
    for (int vi = M.vfirst[m]; vi < M.vfirst[m + 1]; ++vi) {
        const int q = M.vsmall[vi], qd = M.vquad[vi];
        face_map2_t(A.fbar + (P.t.fo[eb] + (int64_t)fB * n2) * V, n, res, n, adj_mortar_dir(P, sp, qd, 0, n, true, true),
                    adj_mortar_dir(P, sp, qd, 1, n, true, true), V, sT1);
        fv_layer_t<NK, true>(P, q, fS, n, res, Ub, sT1, sT2);
    }
}


#define DGFV_DISPATCH(nk, call)                          \
    switch (nk) {                                        \
        case 1: { constexpr int NK = 1; call; } break;   \
        case 2: { constexpr int NK = 2; call; } break;   \
        default: { constexpr int NK = 3; call; } break;  \
    }

void launch_adj_mortar_virt(int nk, const Params& P, const AdjBuffers& A, const MortarTables& M, int n_virt,
                            int which, cudaStream_t s) {
    if (n_virt <= 0) return;
    DGFV_DISPATCH(nk, (k_adj_mortar_virt<NK><<<n_virt, 128, 0, s>>>(P, A, M, which)));
}

void launch_adj_mortar_big(int nk, const Params& P, const AdjBuffers& A, const MortarTables& M, int n_mort,
                           int which, cudaStream_t s) {
    if (n_mort <= 0) return;
    DGFV_DISPATCH(nk, (k_adj_mortar_big<NK><<<n_mort, 128, 0, s>>>(P, A, M, which)));
}

void launch_adj_mortar_nb(int nk, const Params& P, const AdjBuffers& A, const MortarTables& M, int n_mort,
                          double* Ub, cudaStream_t s) {
    if (n_mort <= 0) return;
    DGFV_DISPATCH(nk, (k_adj_mortar_nb<NK><<<n_mort, 128, 0, s>>>(P, A, M, Ub)));
}

void launch_adj_surface(int nk, const Params& P, const AdjBuffers& A, const Tiles& T, int ntiles, const double* Rb,
                        cudaStream_t s) {
    if (ntiles <= 0) return;
    DGFV_DISPATCH(nk, (k_adj_surface<NK><<<ntiles, 256, 0, s>>>(P, A, T, Rb)));
}

void launch_adj_faces(int nk, const Params& P, const AdjBuffers& A, const Faces& F, const FaceTiles& conf,
                      int nconf, cudaStream_t s) {
    if (nconf > 0) DGFV_DISPATCH(nk, (k_adj_face_conf<NK><<<nconf, 128, 0, s>>>(P, A, F, conf)));
}

void launch_adj_mixed_faces(int nk, const Params& P, const AdjBuffers& A, const Faces& F, const FaceTiles& T,
                            int ntiles, const int32_t* mface, const int64_t* mpt, int nmixed, double* Sin,
                            double* Sout, cudaStream_t s) {
    if (nmixed <= 0) return;
    DGFV_DISPATCH(nk, (k_adj_mixed_in<NK><<<nmixed, 128, 0, s>>>(P, A, F, mface, mpt, Sin, Sout),
                       k_adj_mixed_point<NK><<<ntiles, 128, 0, s>>>(P, A, F, T, mface, mpt, Sin, Sout),
                       k_adj_mixed_out<NK><<<nmixed, 128, 0, s>>>(P, A, F, mface, mpt, Sin)));
}

size_t adj_volume_smem_bytes(int nk, int n, int count) {
    const int V = nk + 4;
    return sizeof(double) * (size_t)(n * n + 4 * n + count * 3 * V * n * n * n);
}

void launch_adj_vol_a(int nk, const Params& P, const Tiles& T, int ntiles, size_t smem, const double* U,
                      const double* Rb, double* Ub, double* gvol, double* gf, cudaStream_t s, int split) {
    if (ntiles <= 0) return;
    DGFV_DISPATCH(nk, (cudaFuncSetAttribute(k_adj_vol_a<NK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                       k_adj_vol_a<NK><<<ntiles, 256, smem, s>>>(P, T, U, Rb, gf),
                       k_adj_point<NK><<<ntiles, 128, 0, s>>>(P, T, U, gf, Ub, gvol, split)));
}

size_t adj_split_smem_bytes(int nk, int n, int count) {
    const int NT = 6 + nk, n3 = n * n * n;
    return sizeof(double) * (size_t)(n * n + 2 * count * NT * n3);
}

void launch_adj_split(int nk, const Params& P, const Tiles& T, int ntiles, size_t smem, const double* U,
                      const double* Rb, double* Ub, cudaStream_t s) {
    if (ntiles <= 0) return;
    DGFV_DISPATCH(nk, (cudaFuncSetAttribute(k_adj_split<NK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                       k_adj_split<NK><<<ntiles, 256, smem, s>>>(P, T, U, Rb, Ub)));
}

void launch_adj_vol_b(int nk, const Params& P, const AdjBuffers& A, const Tiles& T, int ntiles, size_t smem,
                      const double* gvol, double* Ub, cudaStream_t s) {
    if (ntiles <= 0) return;
    DGFV_DISPATCH(nk, (cudaFuncSetAttribute(k_adj_vol_b<NK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                       k_adj_vol_b<NK><<<ntiles, 256, smem, s>>>(P, A, T, gvol, Ub)));
}

void launch_adj_lift(int nk, const Params& P, const AdjBuffers& A, const Faces& F, const int32_t* list, int nfaces,
                     cudaStream_t s) {
    if (nfaces <= 0) return;
    DGFV_DISPATCH(nk, (k_adj_lift<NK><<<nfaces, 64, 0, s>>>(P, A, F, list)));
}

void launch_adj_surface_fv(int nk, const Params& P, const AdjBuffers& A, const Tiles& T, int ntiles, const double* Rb,
                           cudaStream_t s) {
    if (ntiles <= 0) return;
    DGFV_DISPATCH(nk, (k_adj_surface_fv<NK><<<ntiles, 128, 0, s>>>(P, A, T, Rb)));
}

void launch_adj_prolong(int nk, const Params& P, const AdjBuffers& A, const Tiles& T, int ntiles, double* Ub,
                        cudaStream_t s) {
    if (ntiles <= 0) return;
    DGFV_DISPATCH(nk, (k_adj_prolong<NK><<<ntiles, 256, 0, s>>>(P, A, T, Ub)));
}

void launch_axpby(int64_t n, double a, const double* x, double b, const double* y, double* out, cudaStream_t s) {
    if (n <= 0) return;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 32);
    k_axpby<<<blocks, 256, 0, s>>>(n, a, x, b, y, out);
}

void launch_rk3_adj_combine(int64_t n, int mode, double c1, double c2, double dt, const double* x, const double* y,
                            double* o1, double* o2, cudaStream_t s) {
    if (n <= 0) return;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    k_rk3_adj_combine<<<blocks, 256, 0, s>>>(n, mode, c1, c2, dt, x, y, o1, o2);
}

}  // namespace dgfv
