// Volume integrals of the DG elements (sm_103a): the standard weak form
// (Eqs. 22, 23) and the split form on LGL nodes (Sec. 3.5).  Separate from
// kernels.cu so that the point-count instantiations compile in parallel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "device_util.cuh"
#include "kernels.h"

namespace dgfv {

// ---------------------------------------------------------------------------------
// k_dg_volume: tiles of DG elements of one degree; the lifted gradient lives in
// shared memory (3V n^3 doubles per element) and is overwritten in place by
// the nodal fluxes before the volume integral.
// NP > 0: the tile's point count as a compile-time constant (unrolled
// contractions); NP = 0: read from the tile.
template <int NK, int NP>
__device__ __forceinline__ void dg_volume_body(const Params& P, const Tiles& T, const double* __restrict__ U,
                                               int tile) {
    constexpr int V = NK + 4;
    extern __shared__ double sm[];
    const int first = T.first[tile], count = T.count[tile];
    const int n = NP > 0 ? NP : T.n[tile];
    const int n2 = n * n, n3 = n2 * n, q = n2 + 2 * n;
    double* sl = sm;                 // lm, lp (2n)
    double* sS = sl + 2 * n;         // per element and direction: (2/h_d) Dhat, (2/h_d) lhat(-1), (2/h_d) lhat(+1)
    double* sG = sS + count * 3 * q; // count * 3V * n3
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        sl[i] = B(P, P.bi.lm[n])[i];
        sl[n + i] = B(P, P.bi.lp[n])[i];
    }
    for (int i = threadIdx.x; i < count * 3 * q; i += blockDim.x) {
        const int el = i / (3 * q), r = i % (3 * q), d = r / q, k = r % q;
        const double rh = P.t.rh[3 * T.items[first + el] + d];
        const double b = k < n2 ? B(P, P.bi.dhat[n])[k]
                                : (k < n2 + n ? B(P, P.bi.lhm[n])[k - n2] : B(P, P.bi.lhp[n])[k - n2 - n]);
        sS[i] = rh * b;
    }
    __syncthreads();
    const bool visc = P.ph.viscous;
    if (visc) {
        // lifting, Eq. 23 (gradient sign): g^d_v = (2/h_d)(sum_m Dhat_im u_m + lhat_i(1) U*+ - lhat_i(-1) U*-)
        const int per = 3 * V * n3;
        for (int idx = threadIdx.x; idx < count * per; idx += blockDim.x) {
            const int el = idx / per, r = idx % per, d = r / (V * n3), r2 = r % (V * n3), v = r2 / n3, c = r2 % n3;
            const int e = T.items[first + el];
            const int i = c % n, j = (c / n) % n, k = c / n2;
            const int m0 = d == 0 ? i : (d == 1 ? j : k);
            const int a = d == 0 ? j : i, b = d == 2 ? j : k;
            const double* src = U + P.t.off[e] + (int64_t)v * n3;
            const double* Sd = sS + (el * 3 + d) * q;
            double s = 0.0;
            for (int m = 0; m < n; ++m) s = fma(Sd[m0 * n + m], src[node_index(n, d, m, a, b)], s);
            const int64_t fo = P.t.fo[e];
            const int p = a + n * b;
            s = fma(Sd[n2 + n + m0], P.b.flift[(fo + (int64_t)(2 * d + 1) * n2) * V + v * n2 + p], s);
            s = fma(-Sd[n2 + m0], P.b.flift[(fo + (int64_t)(2 * d) * n2) * V + v * n2 + p], s);
            sG[el * per + r] = s;
        }
        __syncthreads();
        // traces of the gradient on the six faces
        const int pt = 6 * 3 * V * n2;
        for (int idx = threadIdx.x; idx < count * pt; idx += blockDim.x) {
            const int el = idx / pt, r = idx % pt, f = r / (3 * V * n2), r2 = r % (3 * V * n2), x = r2 / n2, p = r2 % n2;
            const int e = T.items[first + el];
            const int d = f >> 1, a = p % n, b = p / n;
            const double* lb = sl + ((f & 1) ? n : 0);
            const double* src = sG + el * 3 * V * n3 + x * n3;
            double s = 0.0;
            for (int m = 0; m < n; ++m) s = fma(lb[m], src[node_index(n, d, m, a, b)], s);
            P.b.fg[(P.t.fo[e] + (int64_t)f * n2) * 3 * V + x * n2 + p] = s;
        }
        __syncthreads();
    }
    // fluxes at the nodes: F_d = F^c_d(u) + F^v_d(u, g), written over g
    for (int idx = threadIdx.x; idx < count * n3; idx += blockDim.x) {
        const int el = idx / n3, c = idx % n3;
        const int e = T.items[first + el];
        const double* src = U + P.t.off[e] + c;
        double u[V];
#pragma unroll
        for (int v = 0; v < V; ++v) u[v] = src[(int64_t)v * n3];
        Prim<NK> s;
        prim<NK>(P.ph, u, s);
        double* G = sG + el * 3 * V * n3 + c;
        PrimGrad<NK> pg;
        if (visc) {
            double g[3 * V];
#pragma unroll
            for (int x = 0; x < 3 * V; ++x) g[x] = G[x * n3];
            prim_grad<NK>(P.ph, s, g, pg);
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double F[V];
            flux_conv<NK>(u, s, d, F);
            if (visc) flux_visc_add<NK>(P.ph, s, pg, d, F);
#pragma unroll
            for (int v = 0; v < V; ++v) G[(d * V + v) * n3] = F[v];
        }
    }
    __syncthreads();
    // volume integral sum_d sum_m (2/h_d) Dhat_{i_d m} F_d(m), one accumulation chain
    const int per = V * n3;
    for (int idx = threadIdx.x; idx < count * per; idx += blockDim.x) {
        const int el = idx / per, r = idx % per, v = r / n3, c = r % n3;
        const int e = T.items[first + el];
        const int ijk[3] = {c % n, (c / n) % n, c / n2};
        const double* Fe = sG + el * 3 * V * n3;
        double acc = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int m0 = ijk[d];
            const int a = d == 0 ? ijk[1] : ijk[0], b = d == 2 ? ijk[1] : ijk[2];
            const double* src = Fe + (d * V + v) * n3;
            const double* Sd = sS + (el * 3 + d) * q + m0 * n;
            for (int m = 0; m < n; ++m) acc = fma(Sd[m], src[node_index(n, d, m, a, b)], acc);
        }
        P.b.rtmp[P.t.off[e] + r] = acc;
    }
}

template <int NK>
__device__ __forceinline__ void dg_volume_tile(const Params& P, const Tiles& T, const double* __restrict__ U,
                                               int tile) {
    switch (T.n[tile]) {
        case 2: dg_volume_body<NK, 2>(P, T, U, tile); break;
        case 3: dg_volume_body<NK, 3>(P, T, U, tile); break;
        case 4: dg_volume_body<NK, 4>(P, T, U, tile); break;
        case 5: dg_volume_body<NK, 5>(P, T, U, tile); break;
        case 6: dg_volume_body<NK, 6>(P, T, U, tile); break;
        case 7: dg_volume_body<NK, 7>(P, T, U, tile); break;
        default: dg_volume_body<NK, 8>(P, T, U, tile); break;
    }
}

template <int NK, int MINB>
__global__ void __launch_bounds__(256, MINB) k_dg_volume(Params P, Tiles T, const double* __restrict__ U) {
    dg_volume_tile<NK>(P, T, U, blockIdx.x);
}

// Persistent form: as many CTAs as fit on the GPU at once, each taking tiles
// (of one degree each, every degree in the one launch) from a work queue, the
// costliest degrees first (the tiles are stored by increasing point count and
// taken from the end).  The queue is a counter the launch sets to zero; every
// CTA stops once the counter passes the last tile, so the loop runs at most
// ntiles times and never waits on another CTA.
template <int NK, int MINB>
__global__ void __launch_bounds__(256, MINB) k_dg_volume_persistent(Params P, Tiles T, const double* __restrict__ U,
                                                                    int ntiles, int* __restrict__ queue) {
    __shared__ int s_next;
    for (int it = 0; it < ntiles; ++it) {
        if (threadIdx.x == 0) s_next = atomicAdd(queue, 1);
        __syncthreads();
        const int t = s_next;
        if (t >= ntiles) break;
        dg_volume_tile<NK>(P, T, U, ntiles - 1 - t);
        __syncthreads();  // the tile's shared memory and s_next are reused
    }
}

// ---------------------------------------------------------------------------------
// k_dg_volume_split: split-form DGSEM on LGL nodes (Sec. 3.5).  Lifting and
// gradient traces as in k_dg_volume; the nodal viscous fluxes overwrite the
// gradient; the volume term of node i along direction d is
//   sum_m Dhat_im F^v_d(m) + sum_m S_im F#_d(u_i, u_m),   S = 2D - W^{-1}B,
// F# the kinetic-energy-preserving two-point flux (its diagonal F#(u_i,u_i) =
// F^c(u_i) carries the boundary correction).  One thread per node, all variables.
template <int NK, int NP>
__device__ __forceinline__ void dg_volume_split_body(const Params& P, const Tiles& T, const double* __restrict__ U) {
    constexpr int V = NK + 4, NT = 6 + NK;
    extern __shared__ double sm[];
    const int first = T.first[blockIdx.x], count = T.count[blockIdx.x];
    const int n = NP > 0 ? NP : T.n[blockIdx.x];
    const int n2 = n * n, n3 = n2 * n;
    const bool visc = P.ph.viscous;
    double* sD = sm;            // n*n Dhat
    double* sS = sD + n * n;    // n*n split matrix
    double* sl = sS + n * n;    // lm, lp, lhm, lhp (4n)
    double* sK = sl + 4 * n;    // count * NT * n3 two-point flux tuples
    double* sG = sK + count * NT * n3;  // count * 3V * n3: g, then F^v, then the per-direction partial sums
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
        sD[i] = B(P, P.bi.dhat[n])[i];
        sS[i] = B(P, P.bi.dsplit[n])[i];
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        sl[i] = B(P, P.bi.lm[n])[i];
        sl[n + i] = B(P, P.bi.lp[n])[i];
        sl[2 * n + i] = B(P, P.bi.lhm[n])[i];
        sl[3 * n + i] = B(P, P.bi.lhp[n])[i];
    }
    __syncthreads();
    if (visc) {
        // lifting, Eq. 23 (gradient sign), as in k_dg_volume
        const int per = 3 * V * n3;
        for (int idx = threadIdx.x; idx < count * per; idx += blockDim.x) {
            const int el = idx / per, r = idx % per, d = r / (V * n3), r2 = r % (V * n3), v = r2 / n3, c = r2 % n3;
            const int e = T.items[first + el];
            const int i = c % n, j = (c / n) % n, k = c / n2;
            const int m0 = d == 0 ? i : (d == 1 ? j : k);
            const int a = d == 0 ? j : i, b = d == 2 ? j : k;
            const double* src = U + P.t.off[e] + (int64_t)v * n3;
            double s = 0.0;
            for (int m = 0; m < n; ++m) s = fma(sD[m0 * n + m], src[node_index(n, d, m, a, b)], s);
            const int64_t fo = P.t.fo[e];
            const int p = a + n * b;
            s = fma(sl[3 * n + m0], P.b.flift[(fo + (int64_t)(2 * d + 1) * n2) * V + v * n2 + p], s);
            s = fma(-sl[2 * n + m0], P.b.flift[(fo + (int64_t)(2 * d) * n2) * V + v * n2 + p], s);
            sG[el * per + r] = P.t.rh[3 * e + d] * s;
        }
        __syncthreads();
        const int pt = 6 * 3 * V * n2;
        for (int idx = threadIdx.x; idx < count * pt; idx += blockDim.x) {
            const int el = idx / pt, r = idx % pt, f = r / (3 * V * n2), r2 = r % (3 * V * n2), x = r2 / n2, p = r2 % n2;
            const int e = T.items[first + el];
            const int d = f >> 1, a = p % n, b = p / n;
            const double* lb = sl + ((f & 1) ? n : 0);
            const double* src = sG + el * 3 * V * n3 + x * n3;
            double s = 0.0;
            for (int m = 0; m < n; ++m) s = fma(lb[m], src[node_index(n, d, m, a, b)], s);
            P.b.fg[(P.t.fo[e] + (int64_t)f * n2) * 3 * V + x * n2 + p] = s;
        }
        __syncthreads();
    }
    // per node: two-point flux tuple; viscous fluxes written over the gradient
    for (int idx = threadIdx.x; idx < count * n3; idx += blockDim.x) {
        const int el = idx / n3, c = idx % n3;
        const int e = T.items[first + el];
        const double* src = U + P.t.off[e] + c;
        double u[V];
#pragma unroll
        for (int v = 0; v < V; ++v) u[v] = src[(int64_t)v * n3];
        Prim<NK> s;
        prim<NK>(P.ph, u, s);
        double t[NT];
        kep_tuple<NK>(s, t);
#pragma unroll
        for (int q = 0; q < NT; ++q) sK[(el * NT + q) * n3 + c] = t[q];
        if (visc) {
            double* G = sG + el * 3 * V * n3 + c;
            double g[3 * V];
#pragma unroll
            for (int x = 0; x < 3 * V; ++x) g[x] = G[x * n3];
            PrimGrad<NK> pg;
            prim_grad<NK>(P.ph, s, g, pg);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                double Fv[V];
                flux_visc<NK>(P.ph, s, pg, d, Fv);
#pragma unroll
                for (int v = 0; v < V; ++v) G[(d * V + v) * n3] = Fv[v];
            }
        }
    }
    __syncthreads();
    // volume term, one thread per line (element, direction d, line (a, b)):
    // every two-point flux of a pair of the line's nodes once, F#(u_i, u_m) =
    // F#(u_m, u_i), added to both nodes with S_im and S_mi; the viscous part
    // sum_m Dhat_im F^v_d(m) first.  The line's partial sums (times 2/h_d) are
    // written over its F^v_d values (only this thread reads them).
    constexpr int NL = NP > 0 ? NP : MAXP;
    const int lines = 3 * n2;
    for (int idx = threadIdx.x; idx < count * lines; idx += blockDim.x) {
        const int el = idx / lines, r = idx % lines, d = r / n2, p = r % n2, a = p % n, b = p / n;
        const int e = T.items[first + el];
        const double* K = sK + el * NT * n3;
        double* Fv = sG + el * 3 * V * n3 + d * V * n3;
        double acc[NL][V];
#pragma unroll
        for (int i = 0; i < NL; ++i)
#pragma unroll
            for (int v = 0; v < V; ++v) acc[i][v] = 0.0;
        if (visc) {
#pragma unroll
            for (int i = 0; i < NL; ++i)
#pragma unroll
                for (int m = 0; m < NL; ++m) {
                    const double Dim = sD[i * n + m];
                    const int cm = node_index(n, d, m, a, b);
#pragma unroll
                    for (int v = 0; v < V; ++v) acc[i][v] = fma(Dim, Fv[v * n3 + cm], acc[i][v]);
                }
        }
#pragma unroll
        for (int i = 0; i < NL; ++i) {
            const int ci = node_index(n, d, i, a, b);
            double ti[NT], F[V];
#pragma unroll
            for (int q = 0; q < NT; ++q) ti[q] = K[q * n3 + ci];
            kep_flux<NK>(ti, ti, d, F);  // = F^c(u_i)
            const double Sii = sS[i * n + i];
#pragma unroll
            for (int v = 0; v < V; ++v) acc[i][v] = fma(Sii, F[v], acc[i][v]);
#pragma unroll
            for (int m = i + 1; m < NL; ++m) {
                const int cm = node_index(n, d, m, a, b);
                double tm[NT];
#pragma unroll
                for (int q = 0; q < NT; ++q) tm[q] = K[q * n3 + cm];
                kep_flux<NK>(ti, tm, d, F);
                const double Sim = sS[i * n + m], Smi = sS[m * n + i];
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    acc[i][v] = fma(Sim, F[v], acc[i][v]);
                    acc[m][v] = fma(Smi, F[v], acc[m][v]);
                }
            }
        }
        const double rh = P.t.rh[3 * e + d];
#pragma unroll
        for (int i = 0; i < NL; ++i) {
            const int ci = node_index(n, d, i, a, b);
#pragma unroll
            for (int v = 0; v < V; ++v) Fv[v * n3 + ci] = rh * acc[i][v];
        }
    }
    __syncthreads();
    // sum of the three directions
    const int per = V * n3;
    for (int idx = threadIdx.x; idx < count * per; idx += blockDim.x) {
        const int el = idx / per, r = idx % per;
        const int e = T.items[first + el];
        const double* G = sG + el * 3 * V * n3 + r;
        P.b.rtmp[P.t.off[e] + r] = G[0] + G[V * n3] + G[2 * V * n3];
    }
}

template <int NK>
__global__ void __launch_bounds__(256) k_dg_volume_split(Params P, Tiles T, const double* __restrict__ U) {
    switch (T.n[blockIdx.x]) {  // the tile's point count as a compile-time constant
        case 2: dg_volume_split_body<NK, 2>(P, T, U); break;
        case 3: dg_volume_split_body<NK, 3>(P, T, U); break;
        case 4: dg_volume_split_body<NK, 4>(P, T, U); break;
        case 5: dg_volume_split_body<NK, 5>(P, T, U); break;
        case 6: dg_volume_split_body<NK, 6>(P, T, U); break;
        case 7: dg_volume_split_body<NK, 7>(P, T, U); break;
        default: dg_volume_split_body<NK, 8>(P, T, U); break;
    }
}

// ================================================================= launchers
#define DGFV_DISPATCH(nk, call)           \
    switch (nk) {                         \
        case 1: { constexpr int NK = 1; call; } break; \
        case 2: { constexpr int NK = 2; call; } break; \
        default: { constexpr int NK = 3; call; } break; \
    }

size_t volume_smem_bytes(int nk, int n, int count) {
    const int V = nk + 4;
    return sizeof(double) * (size_t)(2 * n + count * 3 * (n * n + 2 * n) + count * 3 * V * n * n * n);
}

// variant bit 0: 128 threads per CTA (else 256); bit 1: register budget for
// three 256-thread CTAs per SM (else two).
void launch_dg_volume(int nk, const Params& P, const Tiles& T, int ntiles, size_t smem, const double* U,
                      cudaStream_t s, int variant) {
    if (ntiles <= 0) return;
    const int threads = (variant & 1) ? 128 : 256;
    if (variant & 2) {
        DGFV_DISPATCH(nk, (cudaFuncSetAttribute(k_dg_volume<NK, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)smem),
                           k_dg_volume<NK, 3><<<ntiles, threads, smem, s>>>(P, T, U)));
    } else {
        DGFV_DISPATCH(nk, (cudaFuncSetAttribute(k_dg_volume<NK, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)smem),
                           k_dg_volume<NK, 2><<<ntiles, threads, smem, s>>>(P, T, U)));
    }
}

void launch_dg_volume_persistent(int nk, const Params& P, const Tiles& T, int ntiles, size_t smem, const double* U,
                                 cudaStream_t s, int variant, int* queue, int n_sm) {
    if (ntiles <= 0) return;
    const int threads = (variant & 1) ? 128 : 256;
    cudaMemsetAsync(queue, 0, sizeof(int), s);
    int per_sm = 1;
    if (variant & 2) {
        DGFV_DISPATCH(nk, (cudaFuncSetAttribute(k_dg_volume_persistent<NK, 3>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                           cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dg_volume_persistent<NK, 3>,
                                                                         threads, smem),
                           k_dg_volume_persistent<NK, 3><<<std::min(ntiles, std::max(1, per_sm) * n_sm), threads,
                                                           smem, s>>>(P, T, U, ntiles, queue)));
    } else {
        DGFV_DISPATCH(nk, (cudaFuncSetAttribute(k_dg_volume_persistent<NK, 2>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                           cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dg_volume_persistent<NK, 2>,
                                                                         threads, smem),
                           k_dg_volume_persistent<NK, 2><<<std::min(ntiles, std::max(1, per_sm) * n_sm), threads,
                                                           smem, s>>>(P, T, U, ntiles, queue)));
    }
}

size_t volume_split_smem_bytes(int nk, int n, int count, bool viscous) {
    (void)viscous;  // the per-direction partial sums need the 3V n^3 block either way
    const int V = nk + 4, NT = 6 + nk;
    return sizeof(double) * (size_t)(2 * n * n + 4 * n + count * (NT + 3 * V) * n * n * n);
}

void launch_dg_volume_split(int nk, const Params& P, const Tiles& T, int ntiles, size_t smem, const double* U,
                            cudaStream_t s) {
    if (ntiles <= 0) return;
    DGFV_DISPATCH(nk, (cudaFuncSetAttribute(k_dg_volume_split<NK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem),
                       k_dg_volume_split<NK><<<ntiles, 256, smem, s>>>(P, T, U)));
}

}  // namespace dgfv
