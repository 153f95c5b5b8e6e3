// Adjoint of the FV sub-cell operator (Sec. 3.1.2: the second-order
// finite-volume scheme on N_FV^3 sub-cells with the minmod-limited
// reconstruction of the reconstruction variables, central-difference
// gradients and the sub-cell face fluxes) for the FV elements of a frozen
// hybrid pattern, and the gather of the neighbour-layer adjoints.
//
//   k_adj_fv         one CTA per FV element: recomputes the forward
//                    quantities of k_fv and runs its steps backwards
//   k_adj_fv_gather  U_bar of every element += (its layers seen by FV
//                    neighbours)^T
#include <cuda_runtime.h>

#include "adjoint.h"
#include "common.cuh"
#include "device_util.cuh"
#include "physics_adj.cuh"

namespace dgfv {

// Shared-memory layout of k_adj_fv, in doubles.  GS = 1 keeps the
// central-difference gradients of the element's sub-cells (3V n^3), formed
// once, and turns the conservative means into reconstruction variables in
// place (the conservative means are read again from U at the end); GS = 0
// forms a sub-cell's gradient at each of its faces.  The neighbour gather's
// scratch lies over the regions filled after the gather (G; W and Nw).
struct AdjFvLayout {
    int g, u, w, nb, nw, t, total;
};

__host__ __device__ inline AdjFvLayout adj_fv_layout(int V, int n, int gs) {
    const int n2 = n * n, n3 = n2 * n, tmp = 6 * V * (MAXP * MAXP + n * MAXP);
    AdjFvLayout L;
    if (gs) {  // [ G | U -> W | Nb | Nw ]
        const int gsz = 3 * V * n3 > tmp ? 3 * V * n3 : tmp;
        L.g = 0;
        L.t = 0;
        L.u = gsz;
        L.w = gsz;
        L.nb = L.u + V * n3;
        L.nw = L.nb + 6 * V * n2;
        L.total = L.nw + 6 * V * n2;
    } else {  // [ U | Nb | W | Nw ]
        L.g = 0;
        L.u = 0;
        L.nb = V * n3;
        L.w = L.nb + 6 * V * n2;
        L.nw = L.w + V * n3;
        L.t = L.w;
        L.total = L.w + (V * n3 + 6 * V * n2 > tmp ? V * n3 + 6 * V * n2 : tmp);
    }
    return L;
}

// k_adj_fv: one CTA per FV element, after the face and lifting adjoints (which
// leave the adjoints of the element's reconstructed face states in ubar and of
// its boundary-cell gradients in gbar).  Recomputes the forward quantities of
// k_fv (neighbour values, reconstruction variables, slopes, gradients) and
// runs its steps backwards:
//   1. interior sub-cell faces: F_bar = (n/h_d)(R_bar(c_R) - R_bar(c_L)), the
//      point-flux reverse gives the adjoints of the two reconstructed states and
//      of the two cells' gradients;
//   2. element faces: the reconstructed-state and gradient adjoints from ubar, gbar;
//   3. per cell and direction: the limited slope once for both face values
//      (w+- = w_c +- h), w_to_cons^T of both, the slope's reverse along the
//      branch the forward took (minmod), and gradient^T (central
//      differences); contributions beyond the element go to the neighbour
//      values;
//   4. cons_to_w^T: the element's U_bar (written), and the neighbour values'
//      adjoints in conservative variables, left in the element's fbar slots for
//      k_adj_fv_gather.
// The reconstructed values and their states follow k_fv's arithmetic (a half
// slope minmod(dw-, dw+)/2 inside the element, l/2 minmod(dw-/dist-,
// dw+/dist+) in the boundary sub-cells; face_state).  Scratch in global
// memory, in the element's own regions of the adjoint buffers the DG kernels
// do not use for FV elements:
// rec_bar (6V n^3) in gf, grad_bar (3V n^3) in gvol, w_bar and the direct
// u_bar (2 x V n^3) in fvs; the neighbour adjoints in the element's sbar
// (reconstruction variables) and fbar (conservative) face slots.  Sums over
// several writers use atomics.  Launched with 128 threads (two CTAs per SM)
// where the layout allows two, else 256.
template <int NK, int GS>
__global__ void __launch_bounds__(256) k_adj_fv(Params P, AdjBuffers A, Tiles T, const double* __restrict__ U,
                                               const double* __restrict__ Rb, double* __restrict__ Ub,
                                               double* __restrict__ gf, double* __restrict__ gvol,
                                               double* __restrict__ fvs, int64_t cap_state) {
    constexpr int V = NK + 4;
    extern __shared__ double sm[];
    const int e = T.items[T.first[blockIdx.x]];
    const int n = P.t.n[e], n2 = n * n, n3 = n2 * n;  // this element's sub-cells (the shared memory fits the largest)
    const AdjFvLayout L = adj_fv_layout(V, n, GS);
    double* sU = sm + L.u;    // V n3 conservative means (GS = 1: turned into sW in place)
    double* sW = sm + L.w;    // V n3 reconstruction variables
    double* sNb = sm + L.nb;  // 6 V n2 neighbour values (conservative)
    double* sNw = sm + L.nw;  // 6 V n2 neighbour reconstruction variables
    double* sG = sm + L.g;    // 3V n3 gradients (GS = 1)
    __shared__ double sID[6], sGS[6];
    __shared__ const double* sMap[6];
    __shared__ int sNq[6];
    const int64_t off = P.t.off[e];
    const double* rh = P.t.rh + 3 * e;
    const double l = 2.0 / n, il = 0.5 * n;
    const bool visc = P.ph.viscous;
    double* recb = gf + 6 * off;             // [d][side][v][c]: 6 V n3
    double* gradb = gvol + 3 * off;          // [x][c]: 3V n3
    double* wbar = fvs + off;                // V n3
    double* ubc = fvs + cap_state + off;     // V n3
    double* nbwb = A.sbar + P.t.fo[e] * V;   // 6 slots of V n2
    double* nbub = A.fbar + P.t.fo[e] * V;   // 6 slots of V n2
    for (int i = threadIdx.x; i < V * n3; i += blockDim.x) {
        sU[i] = U[off + i];
        wbar[i] = 0.0;
        ubc[i] = 0.0;
    }
    for (int i = threadIdx.x; i < 3 * V * n3; i += blockDim.x) gradb[i] = 0.0;
    for (int i = threadIdx.x; i < 6 * V * n2; i += blockDim.x) {
        nbwb[i] = 0.0;
        nbub[i] = 0.0;
    }
    fv_gather_neighbours<NK>(P, U, e, n, sNb, sm + L.t, sID, sGS, sMap, sNq);
    auto cellU = [&](int d, int m, int a, int b, int v) -> double {
        if (m < 0) return sNb[((2 * d) * V + v) * n2 + a + n * b];
        if (m >= n) return sNb[((2 * d + 1) * V + v) * n2 + a + n * b];
        return sU[v * n3 + node_index(n, d, m, a, b)];
    };
    auto grad = [&](int i, int j, int k, double* g) {
        const int c3[3] = {i, j, k};
#pragma unroll
        for (int dd = 0; dd < 3; ++dd) {
            const int m = c3[dd];
            const int a = dd == 0 ? j : i, b = dd == 2 ? j : k;
            const double sc = m == 0 ? sGS[2 * dd] : (m == n - 1 ? sGS[2 * dd + 1] : 0.5 * n * 0.5 * rh[dd]);
#pragma unroll
            for (int v = 0; v < V; ++v)
                g[dd * V + v] = (cellU(dd, m + 1, a, b, v) - cellU(dd, m - 1, a, b, v)) * sc;
        }
    };
    // gradients (GS = 1), reconstruction variables of the cells and of the neighbour layers
    if (GS && visc) {
        for (int c = threadIdx.x; c < n3; c += blockDim.x) {
            double g[3 * V];
            grad(c % n, (c / n) % n, c / n2, g);
#pragma unroll
            for (int x = 0; x < 3 * V; ++x) sG[x * n3 + c] = g[x];
        }
    }
    if (GS) __syncthreads();  // the means are overwritten by W below
    for (int c = threadIdx.x; c < n3; c += blockDim.x) {
        double u[V], w[V];
#pragma unroll
        for (int v = 0; v < V; ++v) u[v] = sU[v * n3 + c];
        cons_to_w<NK>(P.ph, u, w);
#pragma unroll
        for (int v = 0; v < V; ++v) sW[v * n3 + c] = w[v];
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
    __syncthreads();
    auto cellW = [&](int d, int m, int a, int b, int v) -> double {
        if (m < 0) return sNw[((2 * d) * V + v) * n2 + a + n * b];
        if (m >= n) return sNw[((2 * d + 1) * V + v) * n2 + a + n * b];
        return sW[v * n3 + node_index(n, d, m, a, b)];
    };
    // reconstructed reconstruction variables of cell m (along d) at its face side, as k_fv forms them
    auto reconw = [&](int d, int m, int a, int b, int side, double* w) {
        const bool inner = m > 0 && m < n - 1;
        const double ilm = m > 0 ? il : sID[2 * d], ilp = m < n - 1 ? il : sID[2 * d + 1];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const double wc = cellW(d, m, a, b, v);
            const double dm = wc - cellW(d, m - 1, a, b, v), dp = cellW(d, m + 1, a, b, v) - wc;
            const double h = inner ? 0.5 * minmod_bits(dm, dp) : (0.5 * l) * minmod_bits(dm * ilm, dp * ilp);
            w[v] = side > 0 ? wc + h : wc - h;
        }
    };
    auto coords = [&](int d, int m, int a, int b, int& i, int& j, int& k) {
        if (d == 0) { i = m; j = a; k = b; }
        else if (d == 1) { i = a; j = m; k = b; }
        else { i = a; j = b; k = m; }
    };
    // 1. interior sub-cell faces
    const int nif = (n - 1) * n2;
    for (int t = threadIdx.x; t < 3 * nif; t += blockDim.x) {
        const int d = t / nif, fidx = t - d * nif;
        const int m = fidx % (n - 1), p = fidx / (n - 1), a = p % n, b = p / n;
        const int cL = node_index(n, d, m, a, b), cR = node_index(n, d, m + 1, a, b);
        double uL[V], uR[V], Fb[V];
        double uLb[V] = {}, uRb[V] = {};
        Prim<NK> sL, sR;  // as k_fv forms them (face_state: one division each)
        {
            double w[V];
            reconw(d, m, a, b, +1, w);
            face_state<NK>(P.ph, w, uL, sL);
            reconw(d, m + 1, a, b, -1, w);
            face_state<NK>(P.ph, w, uR, sR);
        }
        const double sc = 0.5 * n * rh[d];
#pragma unroll
        for (int v = 0; v < V; ++v) Fb[v] = sc * (Rb[off + (int64_t)v * n3 + cR] - Rb[off + (int64_t)v * n3 + cL]);
        // viscous sides one after the other: a cell's gradient is read (or
        // formed) just before its reverse and its adjoint summed into gradb
        // right after
        auto getg = [&](int side, double* g) {
            if (GS) {
                const int c = side ? cR : cL;
#pragma unroll
                for (int x = 0; x < 3 * V; ++x) g[x] = sG[x * n3 + c];
            } else {
                int i, j, k;
                coords(d, m + side, a, b, i, j, k);
                grad(i, j, k, g);
            }
        };
        auto putgb = [&](int side, const double* gb) {
            const int c = side ? cR : cL;
#pragma unroll
            for (int x = 0; x < 3 * V; ++x) atomicAdd(&gradb[x * n3 + c], gb[x]);
        };
        // the face direction as a compile-time constant: the viscous reverse of
        // the other two directions' gradient entries reduces to the nonzero ones
        if (d == 0)
            face_point_rev_seq_s<NK, 0>(P.ph, uL, sL, uR, sR, 0, Fb, uLb, uRb, true, getg, putgb);
        else if (d == 1)
            face_point_rev_seq_s<NK, 1>(P.ph, uL, sL, uR, sR, 1, Fb, uLb, uRb, true, getg, putgb);
        else
            face_point_rev_seq_s<NK, 2>(P.ph, uL, sL, uR, sR, 2, Fb, uLb, uRb, true, getg, putgb);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            recb[((2 * d + 1) * V + v) * n3 + cL] = uLb[v];  // side + of the left cell
            recb[((2 * d) * V + v) * n3 + cR] = uRb[v];      // side - of the right cell
        }
    }
    // 2. element faces: the face kernels' adjoints of the reconstructed face state and boundary gradient
    for (int i = threadIdx.x; i < 6 * n2; i += blockDim.x) {
        const int f = i / n2, p = i % n2, d = f >> 1, s = f & 1;
        const int c = node_index(n, d, s ? n - 1 : 0, p % n, p / n);
        const int64_t slot = P.t.fo[e] + (int64_t)f * n2;
#pragma unroll
        for (int v = 0; v < V; ++v) recb[(f * V + v) * n3 + c] = A.ubar[slot * V + v * n2 + p];
        if (visc)
#pragma unroll
            for (int x = 0; x < 3 * V; ++x) atomicAdd(&gradb[x * n3 + c], A.gbar[slot * 3 * V + x * n2 + p]);
    }
    __syncthreads();
    // 3. per cell and direction: the slope once, both face values' w_to_cons^T,
    // the slope's reverse along the forward's minmod branch, gradient^T
    auto add_w = [&](int d, int m, int a, int b, int v, double x) {
        if (m < 0) atomicAdd(&nbwb[((2 * d) * V + v) * n2 + a + n * b], x);
        else if (m >= n) atomicAdd(&nbwb[((2 * d + 1) * V + v) * n2 + a + n * b], x);
        else atomicAdd(&wbar[v * n3 + node_index(n, d, m, a, b)], x);
    };
    auto add_u = [&](int d, int m, int a, int b, int v, double x) {
        if (m < 0) atomicAdd(&nbub[((2 * d) * V + v) * n2 + a + n * b], x);
        else if (m >= n) atomicAdd(&nbub[((2 * d + 1) * V + v) * n2 + a + n * b], x);
        else atomicAdd(&ubc[v * n3 + node_index(n, d, m, a, b)], x);
    };
    for (int t = threadIdx.x; t < 3 * n3; t += blockDim.x) {
        const int d = t / n3, c = t % n3;
        const int ijk[3] = {c % n, (c / n) % n, c / n2};
        const int m = ijk[d];
        const int a = d == 0 ? ijk[1] : ijk[0], b = d == 2 ? ijk[1] : ijk[2];
        const bool inner = m > 0 && m < n - 1;
        const double ilm = m > 0 ? il : sID[2 * d], ilp = m < n - 1 ? il : sID[2 * d + 1];
        // h = cs minmod(ga, gb), ga = am dw-, gb = ap dw+ (am = ap = 1, cs = 1/2 inside the element)
        const double cs = inner ? 0.5 : 0.5 * l, am = inner ? 1.0 : ilm, ap = inner ? 1.0 : ilp;
        double wp[V], wm[V], wpb[V] = {}, wmb[V] = {}, rp[V], rm[V];
        unsigned br = 0;  // per variable 2 bits: 1 slope from the minus side, 2 from the plus side
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const double wc = cellW(d, m, a, b, v);
            const double ga = (wc - cellW(d, m - 1, a, b, v)) * am, gb = (cellW(d, m + 1, a, b, v) - wc) * ap;
            double h = 0.0;
            if (ga * gb > 0.0) {
                const bool lo = fabs(ga) <= fabs(gb);
                h = lo ? ga : gb;
                br |= (lo ? 1u : 2u) << (2 * v);
            }
            h *= cs;
            wp[v] = wc + h;
            wm[v] = wc - h;
            rp[v] = recb[((2 * d + 1) * V + v) * n3 + c];
            rm[v] = recb[((2 * d) * V + v) * n3 + c];
        }
        w_to_cons_rev<NK>(P.ph, wp, rp, wpb);
        w_to_cons_rev<NK>(P.ph, wm, rm, wmb);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            // w+- = wc +- h
            const double hb = wpb[v] - wmb[v];
            double own = wpb[v] + wmb[v];
            const unsigned bv = (br >> (2 * v)) & 3u;
            if (bv == 1u) {
                const double x = hb * (cs * am);
                own += x;
                add_w(d, m - 1, a, b, v, -x);
            } else if (bv == 2u) {
                const double x = hb * (cs * ap);
                own -= x;
                add_w(d, m + 1, a, b, v, x);
            }
            add_w(d, m, a, b, v, own);
        }
        if (visc) {
            // g_d(c) = (u(m+1) - u(m-1)) sc
            const double sc = m == 0 ? sGS[2 * d] : (m == n - 1 ? sGS[2 * d + 1] : 0.5 * n * 0.5 * rh[d]);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const double g = gradb[(d * V + v) * n3 + c] * sc;
                add_u(d, m + 1, a, b, v, g);
                add_u(d, m - 1, a, b, v, -g);
            }
        }
    }
    __syncthreads();
    // 4. cons_to_w^T: the element's U_bar and the neighbour values' adjoints
    for (int c = threadIdx.x; c < n3; c += blockDim.x) {
        double u[V], wb[V], ub[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            u[v] = GS ? U[off + (int64_t)v * n3 + c] : sU[v * n3 + c];
            wb[v] = wbar[v * n3 + c];
            ub[v] = ubc[v * n3 + c];
        }
        cons_to_w_rev<NK>(P.ph, u, wb, ub);
#pragma unroll
        for (int v = 0; v < V; ++v) Ub[off + (int64_t)v * n3 + c] = ub[v];
    }
    for (int i = threadIdx.x; i < 6 * n2; i += blockDim.x) {
        const int f = i / n2, p = i % n2;
        double u[V], wb[V], ub[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            u[v] = sNb[(f * V + v) * n2 + p];
            wb[v] = nbwb[(f * V + v) * n2 + p];
            ub[v] = nbub[(f * V + v) * n2 + p];
        }
        cons_to_w_rev<NK>(P.ph, u, wb, ub);
#pragma unroll
        for (int v = 0; v < V; ++v) nbub[(f * V + v) * n2 + p] = ub[v];
    }
}

// k_adj_fv_gather: one CTA per element q; for every face of q with an FV
// element e across, U_bar(q) += layer^T (the adjoint of the layer e read from q,
// left by k_adj_fv in e's fbar slot facing q).
template <int NK>
__global__ void __launch_bounds__(128) k_adj_fv_gather(Params P, AdjBuffers A, double* __restrict__ Ub) {
    constexpr int V = NK + 4;
    __shared__ double sT1[V * MAXP * MAXP], sT2[V * MAXP * MAXP];
    const int q = blockIdx.x;
    for (int fq = 0; fq < 6; ++fq) {
        const int e = P.t.nb[6 * q + fq];
        if (e < 0 || !P.t.fv[e]) continue;
        const int n = P.t.n[e];  // the layer is on e's sub-cell grid
        const double* lb = A.fbar + (P.t.fo[e] + (int64_t)(fq ^ 1) * n * n) * V;
        fv_layer_t<NK>(P, q, fq, n, lb, Ub, sT1, sT2);
    }
}

#define DGFV_DISPATCH(nk, call)                          \
    switch (nk) {                                        \
        case 1: { constexpr int NK = 1; call; } break;   \
        case 2: { constexpr int NK = 2; call; } break;   \
        default: { constexpr int NK = 3; call; } break;  \
    }

// 228 KB of shared memory per SM, 1 KB of it reserved per resident CTA
static bool adj_fv_fits(size_t sm, int ctas) { return ctas * (sm + 1024 + 256) <= 228 * 1024; }

// Layout and block size of k_adj_fv: the gradients kept where two CTAs of 128
// threads fit with them, else formed at each face (two CTAs of 128 threads,
// or one of 256 where only one fits).
static void adj_fv_config(int nk, int nfv, int& gs, int& tpb, size_t& sm) {
    const int V = nk + 4;
    const size_t s1 = sizeof(double) * (size_t)adj_fv_layout(V, nfv, 1).total;
    const size_t s0 = sizeof(double) * (size_t)adj_fv_layout(V, nfv, 0).total;
    if (adj_fv_fits(s1, 2)) {
        gs = 1, tpb = 128, sm = s1;
    } else {
        gs = 0, tpb = adj_fv_fits(s0, 2) ? 128 : 256, sm = s0;
    }
}

size_t adj_fv_smem_bytes(int nk, int nfv) {
    int gs, tpb;
    size_t sm;
    adj_fv_config(nk, nfv, gs, tpb, sm);
    return sm;
}

void launch_adj_fv_elements(int nk, const Params& P, const AdjBuffers& A, const Tiles& T, int ntiles,
                            const double* U, const double* Rb, double* Ub, double* gf, double* gvol, double* fvs,
                            int64_t cap_state, int n_elem, cudaStream_t s) {
    if (ntiles <= 0) return;
    int gs, tpb;
    size_t sm;
    adj_fv_config(nk, P.nfv, gs, tpb, sm);
    if (gs) {
        DGFV_DISPATCH(nk, (cudaFuncSetAttribute(k_adj_fv<NK, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                           k_adj_fv<NK, 1><<<ntiles, tpb, sm, s>>>(P, A, T, U, Rb, Ub, gf, gvol, fvs, cap_state)));
    } else {
        DGFV_DISPATCH(nk, (cudaFuncSetAttribute(k_adj_fv<NK, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                           k_adj_fv<NK, 0><<<ntiles, tpb, sm, s>>>(P, A, T, U, Rb, Ub, gf, gvol, fvs, cap_state)));
    }
    DGFV_DISPATCH(nk, (k_adj_fv_gather<NK><<<n_elem, 128, 0, s>>>(P, A, Ub)));
}

}  // namespace dgfv
