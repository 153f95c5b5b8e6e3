// FP64 CUDA kernel of the finite-volume sub-cell operator (Sec. 3.1.2) of the
// hybrid DG/FV right-hand side (sm_103a), with its shared-memory layouts and
// launch configuration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "device_util.cuh"
#include "kernels.h"

namespace dgfv {

// ---------------------------------------------------------------------------------
// k_fv: one CTA per FV element (n = N_FV sub-cells per direction).
//   neighbour value across each face: FV neighbour -> its boundary sub-cell mean;
//   DG neighbour -> its solution mapped to sub-cell means by V^{DG->FV}, boundary layer.
//   minmod reconstruction of (rho_k, v, p), conservative central-difference
//   gradients, interior sub-cell fluxes -> rtmp; element-face states -> frec, fg.
// The kernel is bound by its FP64 instruction count, so every reconstructed
// face value becomes its conservative and mixture state in one step with a
// single division (face_state), the minmod limiter runs on the integer pipe
// (minmod_bits), and with GS = 1 the central-difference gradient of every
// sub-cell is formed once and kept in shared memory (GS = 0: recomputed at
// each of the cell's faces, for layouts that would not fit).
//
// Shared-memory layout (doubles) of one element, see fv_layout:
//   GS = 1: [gradients 3V n^3 | w V n^3 | neighbour w 6V n^2 | X]; X first holds
//           the conservative means (V n^3) and neighbour values (6V n^2), after
//           the gradients are formed the interior face fluxes 3V (n-1) n^2;
//           the gather's scratch sits in the gradient region.
//   GS = 2: as GS = 1 with the fluxes of two directions in X (the z faces in a
//           second pass), so that two CTAs of 256 threads fit on an SM where
//           GS = 1 fits one of 512 (N_FV = 7 with 2 species: 110.5 KB).
//   GS = 0: [u V n^3 | w V n^3 | neighbour u 6V n^2 | neighbour w 6V n^2 | fluxes],
//           the gather's scratch in the flux region.
template <int NK, int NF, int GS>
__device__ __forceinline__ void fv_body(const Params& P, const Tiles& T, const double* __restrict__ U,
                                        bool faces_only) {
    constexpr int V = NK + 4;
    extern __shared__ double sm[];
    const int n = NF > 0 ? NF : T.n[blockIdx.x], n2 = n * n, n3 = n2 * n;
    const int e = T.items[T.first[blockIdx.x]];
    const FvLayout L = fv_layout(V, n, GS);
    double* sU = sm + L.u;    // V*n3 conservative means
    double* sW = sm + L.w;    // V*n3 reconstruction variables
    double* sNb = sm + L.nb;  // 6*V*n2 neighbour values (conservative)
    double* sNw = sm + L.nw;  // 6*V*n2 neighbour reconstruction variables
    double* sF = sm + L.f;    // 3V*(n-1)*n2 interior face fluxes of the three directions
    double* sG = sm + L.g;    // 3V*n3 gradients (GS = 1)
    double* sT = sm + L.t;    // gather scratch: per face V*MAXP^2 (layer) + V*n*MAXP (half-mapped)
    const int64_t off = P.t.off[e];
    const double* rh = P.t.rh + 3 * e;
    __shared__ double sID[6], sGS[6];  // per face: 1/distance to the neighbour's centre, rh/(l + distance)
    __shared__ const double* sMap[6];
    __shared__ int sNq[6];
    const double l = 2.0 / n, il = 0.5 * n;
    for (int i = threadIdx.x; i < V * n3; i += blockDim.x) sU[i] = U[off + i];
    fv_gather_neighbours<NK>(P, U, e, n, sNb, sT, sID, sGS, sMap, sNq);
    auto cellU = [&](int d, int m, int a, int b, int v) -> double {
        if (m < 0) return sNb[((2 * d) * V + v) * n2 + a + n * b];
        if (m >= n) return sNb[((2 * d + 1) * V + v) * n2 + a + n * b];
        return sU[v * n3 + node_index(n, d, m, a, b)];
    };
    // central-difference gradient of the conservative variables at a cell (coordinates i,j,k)
    auto grad = [&](int i, int j, int k, double* g) {
        const int c3[3] = {i, j, k};
#pragma unroll
        for (int dd = 0; dd < 3; ++dd) {
            const int m = c3[dd];
            const int a = dd == 0 ? j : i, b = dd == 2 ? j : k;
            // 1/(2l) * 2/h = n/(2h) inside; 1/(l + distance) * 2/h at the element boundary
            const double sc = m == 0 ? sGS[2 * dd] : (m == n - 1 ? sGS[2 * dd + 1] : 0.5 * n * 0.5 * rh[dd]);
#pragma unroll
            for (int v = 0; v < V; ++v)
                g[dd * V + v] = (cellU(dd, m + 1, a, b, v) - cellU(dd, m - 1, a, b, v)) * sc;
        }
    };
    for (int c = threadIdx.x; c < n3; c += blockDim.x) {
        double u[V], w[V];
#pragma unroll
        for (int v = 0; v < V; ++v) u[v] = sU[v * n3 + c];
        cons_to_w<NK>(P.ph, u, w);
#pragma unroll
        for (int v = 0; v < V; ++v) sW[v * n3 + c] = w[v];
        if (GS) {
            double g[3 * V];
            grad(c % n, (c / n) % n, c / n2, g);
#pragma unroll
            for (int x = 0; x < 3 * V; ++x) sG[x * n3 + c] = g[x];
        }
    }
    for (int c = threadIdx.x; c < 6 * n2; c += blockDim.x) {
        const int f = c / n2, p = c % n2;
        double u[V], w[V];
#pragma unroll
        for (int v = 0; v < V; ++v) u[v] = sNb[(f * V + v) * n2 + p];
        cons_to_w<NK>(P.ph, u, w);
#pragma unroll
        for (int v = 0; v < V; ++v) sNw[(f * V + v) * n2 + p] = w[v];
    }
    __syncthreads();  // (GS = 1: the means and neighbour values are dead from here on)
    auto cellW = [&](int d, int m, int a, int b, int v) -> double {
        if (m < 0) return sNw[((2 * d) * V + v) * n2 + a + n * b];
        if (m >= n) return sNw[((2 * d + 1) * V + v) * n2 + a + n * b];
        return sW[v * n3 + node_index(n, d, m, a, b)];
    };
    // reconstructed reconstruction variables of cell m (along d) at its face side (-1 or +1):
    // w +- l/2 minmod(dw-/dist-, dw+/dist+); inside the element both distances are l,
    // so the half slope is minmod(dw-, dw+)/2 and w = fma(+-1/2, minmod, w_c) (the
    // same value: halving is exact).  The branch is uniform in the warps of the
    // face pass, which takes the faces between two inner cells first.
    auto face_w = [&](int d, int m, int a, int b, int side, double* w) {
        if (m > 0 && m < n - 1) {
            const int st = d == 0 ? 1 : (d == 1 ? n : n2);  // stride of direction d
            const double* c = sW + node_index(n, d, m, a, b);
            const double hs = side > 0 ? 0.5 : -0.5;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const double wc = c[v * n3];
                const double dm = wc - c[v * n3 - st], dp = c[v * n3 + st] - wc;
                w[v] = fma(hs, minmod_bits(dm, dp), wc);
            }
            return;
        }
        const double ilm = m > 0 ? il : sID[2 * d], ilp = m < n - 1 ? il : sID[2 * d + 1];
        const double hl = side > 0 ? 0.5 * l : -0.5 * l;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const double wc = cellW(d, m, a, b, v);
            const double dm = wc - cellW(d, m - 1, a, b, v), dp = cellW(d, m + 1, a, b, v) - wc;
            w[v] = fma(hl, minmod_bits(dm * ilm, dp * ilp), wc);
        }
    };
    auto cell_grad = [&](int i, int j, int k, double* g) {
        if (GS) {
            const int c = i + n * (j + n * k);
#pragma unroll
            for (int x = 0; x < 3 * V; ++x) g[x] = sG[x * n3 + c];
        } else {
            grad(i, j, k, g);
        }
    };
    auto coords = [&](int d, int m, int a, int b, int& i, int& j, int& k) {
        if (d == 0) { i = m; j = a; k = b; }
        else if (d == 1) { i = a; j = m; k = b; }
        else { i = a; j = b; k = m; }
    };
    // interior sub-cell faces, then the flux differences of every cell
    // (skipped when only the element-face states are wanted: the adjoint's
    // recomputation of the forward face values).  GS = 0, 1: the faces of all
    // three directions in one pass (better balanced over the CTA than one
    // direction at a time); GS = 2: the x and y faces, then the z faces, the
    // flux differences of the first pass kept in the cell's row of rtmp in
    // between (the same sums in the same order, so the same result as GS = 1)
    const int nif = faces_only ? 0 : (n - 1) * n2;
    const int ninner = n > 3 ? (n - 3) * n2 : 0;  // faces m = 1..n-3 of a direction: both cells inner
    constexpr int NPASS = GS == 2 ? 2 : 1;
#pragma unroll 1
    for (int pass = 0; pass < NPASS; ++pass) {
        const int d0 = GS == 2 ? 2 * pass : 0;              // first direction of the pass
        const int nd = GS == 2 ? (pass == 0 ? 2 : 1) : 3;  // directions in the pass
        if (pass > 0) __syncthreads();                      // the first pass's fluxes have been read
        for (int t = threadIdx.x; t < nd * nif; t += blockDim.x) {
            const int dl = t / nif, r = t - dl * nif, d = d0 + dl;
            // work order in a direction: the faces between two inner cells, then
            // the faces m = 0 and m = n-2 (next to a boundary cell)
            int m, p;
            if (r < ninner) {
                m = 1 + r % (n - 3), p = r / (n - 3);
            } else {
                const int q = r - ninner;
                m = q < n2 ? 0 : n - 2, p = q < n2 ? q : q - n2;
            }
            const int a = p % n, b = p / n, fidx = m + (n - 1) * p;
            // F* = F^c*(uL, uR) + (F^v(uL, gL) + F^v(uR, gR))/2, the two viscous
            // fluxes one after the other (one gradient live at a time)
            double uL[V], uR[V], F[V];
            Prim<NK> sL, sR;
            {
                double w[V];
                face_w(d, m, a, b, +1, w);
                face_state<NK>(P.ph, w, uL, sL);
                face_w(d, m + 1, a, b, -1, w);
                face_state<NK>(P.ph, w, uR, sR);
            }
            if (use_roe(P.ph, true))
                riemann_roe<NK>(P.ph, uL, sL, uR, sR, d, F);
            else
                riemann_llf<NK>(uL, sL, uR, sR, d, F);
            if (P.ph.viscous) {
#pragma unroll 1
                for (int side = 0; side < 2; ++side) {
                    int i, j, k;
                    coords(d, m + side, a, b, i, j, k);
                    const int c = i + n * (j + n * k);
                    const int c3[3] = {i, j, k};
                    // d u_v / d x_dd of this cell: kept (GS = 1, 2) or the central difference
                    auto gx = [&](int dd, int v) -> double {
                        if (GS) return sG[(dd * V + v) * n3 + c];
                        const int mm = c3[dd];
                        const int aa = dd == 0 ? c3[1] : c3[0], bb = dd == 2 ? c3[1] : c3[2];
                        const double sc =
                            mm == 0 ? sGS[2 * dd] : (mm == n - 1 ? sGS[2 * dd + 1] : 0.5 * n * 0.5 * rh[dd]);
                        return (cellU(dd, mm + 1, aa, bb, v) - cellU(dd, mm - 1, aa, bb, v)) * sc;
                    };
                    double Fv[V];
                    const Prim<NK>& sx = side ? sR : sL;
                    if (d == 0) flux_visc_dir<NK, 0>(P.ph, sx, gx, Fv);
                    else if (d == 1) flux_visc_dir<NK, 1>(P.ph, sx, gx, Fv);
                    else flux_visc_dir<NK, 2>(P.ph, sx, gx, Fv);
#pragma unroll
                    for (int v = 0; v < V; ++v) F[v] = fma(0.5, Fv[v], F[v]);
                }
            }
#pragma unroll
            for (int v = 0; v < V; ++v) sF[(dl * V + v) * nif + fidx] = F[v];
        }
        __syncthreads();
        for (int c = threadIdx.x; c < (faces_only ? 0 : n3); c += blockDim.x) {
            const int ijk[3] = {c % n, (c / n) % n, c / n2};
            double acc[V];
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] = pass == 0 ? 0.0 : P.b.rtmp[off + (int64_t)v * n3 + c];
#pragma unroll
            for (int dl = 0; dl < nd; ++dl) {
                const int d = d0 + dl, m = ijk[d];
                const int p = (d == 0 ? ijk[1] : ijk[0]) + n * (d == 2 ? ijk[1] : ijk[2]);
                const double sc = 0.5 * n * rh[d];  // n/h_d
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    double t = 0.0;
                    if (m < n - 1) t += sF[(dl * V + v) * nif + m + (n - 1) * p];
                    if (m > 0) t -= sF[(dl * V + v) * nif + (m - 1) + (n - 1) * p];
                    acc[v] = fma(sc, t, acc[v]);
                }
            }
#pragma unroll
            for (int v = 0; v < V; ++v) P.b.rtmp[off + (int64_t)v * n3 + c] = acc[v];
        }
    }
    // element-face states and boundary-cell gradients
    for (int i = threadIdx.x; i < 6 * n2; i += blockDim.x) {
        const int f = i / n2, p = i % n2, a = p % n, b = p / n, d = f >> 1, s = f & 1;
        const int m = s ? n - 1 : 0;
        double w[V], u[V];
        face_w(d, m, a, b, s ? +1 : -1, w);
        w_to_cons<NK>(P.ph, w, u);
        const int64_t slot = P.t.fo[e] + (int64_t)f * n2;
#pragma unroll
        for (int v = 0; v < V; ++v) P.b.frec[slot * V + v * n2 + p] = u[v];
        if (P.ph.viscous) {
            double g[3 * V];
            int ii, jj, kk;
            coords(d, m, a, b, ii, jj, kk);
            cell_grad(ii, jj, kk, g);
#pragma unroll
            for (int x = 0; x < 3 * V; ++x) P.b.fg[slot * 3 * V + x * n2 + p] = g[x];
        }
    }
}


// NF: the sub-cell count as a compile-time constant for the common N_FV = 8,
// a runtime one otherwise (the kernel is bound by its FP64 instructions, which
// a constant count does not change; the integer index work it saves hides
// behind them).  16 warps per SM at 128
// registers a thread: two CTAs of 256 threads where the shared memory of two
// elements fits on an SM, otherwise one CTA of 512 threads.
template <int NK, int TPB, int GS>
__global__ void __launch_bounds__(TPB, 512 / TPB) k_fv(Params P, Tiles T, const double* __restrict__ U,
                                                       int faces_only) {
    if constexpr (GS != 2) {  // GS = 2 never fits two CTAs at N_FV = 8: no body for it
        if (T.n[blockIdx.x] == 8) {
            fv_body<NK, 8, GS>(P, T, U, faces_only != 0);
            return;
        }
    }
    fv_body<NK, 0, GS>(P, T, U, faces_only != 0);
}

#define DGFV_DISPATCH(nk, call)           \
    switch (nk) {                         \
        case 1: { constexpr int NK = 1; call; } break; \
        case 2: { constexpr int NK = 2; call; } break; \
        default: { constexpr int NK = 3; call; } break; \
    }

size_t fv_smem_bytes_variant(int nk, int nfv, int gs) {
    return sizeof(double) * (size_t)fv_layout(nk + 4, nfv, gs).total;
}

// The smaller of the layouts (the one that has to fit for the FV path to run).
size_t fv_smem_bytes(int nk, int nfv) {
    return std::min(fv_smem_bytes_variant(nk, nfv, 0), fv_smem_bytes_variant(nk, nfv, 1));
}

// 228 KB of shared memory per SM, 1 KB of it reserved per resident CTA
static bool fits_per_sm(size_t sm, int ctas) { return ctas * (sm + 1024 + 256) <= 228 * 1024; }

// Layout of the automatic choice: gradients kept with two CTAs of 256 threads
// per SM (GS = 2) where that fits, else with one CTA of 512 (GS = 1), else
// gradients formed at each face (GS = 0).
int fv_variant_auto(int nk, int nfv) {
    if (nfv != 8 && fits_per_sm(fv_smem_bytes_variant(nk, nfv, 2), 2)) return 2;
    return fits_per_sm(fv_smem_bytes_variant(nk, nfv, 1), 1) ? 1 : 0;
}

// variant: 0 automatic, 1 GS = 0, 2 GS = 1, 3 GS = 2 (each where it fits, else
// the automatic choice).
void launch_fv(int nk, const Params& P, const Tiles& T, int ntiles, const double* U, cudaStream_t s, bool faces_only,
               int variant) {
    if (ntiles <= 0) return;
    int gs = variant >= 1 && variant <= 3 ? variant - 1 : fv_variant_auto(nk, P.nfv);
    if (gs == 2 && (P.nfv == 8 || !fits_per_sm(fv_smem_bytes_variant(nk, P.nfv, 2), 2))) gs = fv_variant_auto(nk, P.nfv);
    if (gs == 1 && !fits_per_sm(fv_smem_bytes_variant(nk, P.nfv, 1), 1)) gs = 0;
    const size_t sm = fv_smem_bytes_variant(nk, P.nfv, gs);
    const int fo = faces_only ? 1 : 0;
    if (gs == 2) {
        DGFV_DISPATCH(nk, (cudaFuncSetAttribute(k_fv<NK, 256, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                           k_fv<NK, 256, 2><<<ntiles, 256, sm, s>>>(P, T, U, fo)));
    } else if (gs == 1) {
        DGFV_DISPATCH(nk, (cudaFuncSetAttribute(k_fv<NK, 512, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                           k_fv<NK, 512, 1><<<ntiles, 512, sm, s>>>(P, T, U, fo)));
    } else if (fits_per_sm(sm, 2)) {
        DGFV_DISPATCH(nk, (cudaFuncSetAttribute(k_fv<NK, 256, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                           k_fv<NK, 256, 0><<<ntiles, 256, sm, s>>>(P, T, U, fo)));
    } else {
        DGFV_DISPATCH(nk, (cudaFuncSetAttribute(k_fv<NK, 512, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                           k_fv<NK, 512, 0><<<ntiles, 512, sm, s>>>(P, T, U, fo)));
    }
}

}  // namespace dgfv
