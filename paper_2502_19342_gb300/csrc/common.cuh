// Device-side data layout shared by the kernels and the host driver.
//
// Element tables are structure-of-arrays indexed by element id.  Face data is
// stored per element and face: element e owns 6 face slots of n_e^2 points
// (n_e = N_e+1 nodes for DG, N_FV sub-cells for FV); slot f of e starts at
// face point fo[e] + f*n_e^2 and holds `width` doubles per point as
// [(fo[e] + f*n_e^2)*width + var*n_e^2 + p], p = a + n_e*b with (a, b) the two
// tangential indices in increasing axis order.  Faces: 0:-x 1:+x 2:-y 3:+y 4:-z 5:+z.
#pragma once

#include <cstdint>

#include "physics.cuh"

namespace dgfv {

constexpr int MAXP = 9;        // points per direction of any element (DG: N + 1 <= 8; FV: N_FV <= 9)
constexpr int MAXDG = 8;       // points per direction of a DG element (N <= 7)
constexpr int NBANK = MAXP + 1;

// Offsets (in doubles) of the reference operators in the device bank, indexed
// by the number of points n = N+1 of the DG degree.
struct BankIdx {
    int32_t dhat[NBANK];       // n x n weighted derivative matrix
    int32_t dsplit[NBANK];     // n x n split-form matrix 2D - W^{-1}B (LGL nodes only)
    int32_t w[NBANK];          // quadrature weights of the nodes
    int32_t lm[NBANK], lp[NBANK];    // l_j(-1), l_j(+1)
    int32_t lhm[NBANK], lhp[NBANK];  // l_j(-1)/w_j, l_j(+1)/w_j
    int32_t vinv[NBANK];       // inverse orthonormal-Legendre Vandermonde (n x n)
    int32_t d2f[NBANK][NBANK]; // [n][m] V^{DG->FV}: m sub-cells x n nodes
    int32_t f2d[NBANK][NBANK]; // [n][m] V^{FV->DG}: n x m (pseudo-inverse; L2 projection where m < n)
    int32_t ov[NBANK][NBANK];  // [a][b] sub-cell overlaps, b x a (per-element sub-cell counts)
    int32_t vm[NBANK][NBANK];  // V^{n->m}: m x n (interpolation up, L2 projection down)
    int32_t mi[NBANK][2];      // mortar half s: interpolation to the virtual small side, n x n
    int32_t mp[NBANK][2];      // mortar half s: L2 projection back to the big side, n x n
    int32_t mfi[2], mfp[2];    // the same on N_FV sub-cells
    int32_t eye[NBANK];        // identity, n x n (a face direction that is not halved)
};

struct Tables {
    const uint8_t* n;    // points per direction
    const uint8_t* N;    // DG degree
    const uint8_t* fv;   // FV flag
    const int64_t* off;  // state offset
    const int64_t* fo;   // face-point offset of slot 0
    const int32_t* nb;   // 6 neighbours per element; -1 - slot at a mortar face (Sec. 3.2.3)
    const double* rh;    // 3 per element: 2/h_d
    const double* mnb;   // per mortar slot: V x N_FV^2 FV neighbour values (for FV owners)
    const int32_t* mnbe; // per mortar slot: an element across (its size sets the distance)
};

// Non-conforming interfaces (Sec. 3.2.3).  The virtual small sides of a big
// element face are extra entries n_elem + v of the element tables (no state;
// face slots 0 and 1 only), so that the face kernels couple them with the small
// elements like any other face.  Mortar m: big element, its face fB (0: -x,
// 1: +x), split bits (1: halved along a = y, 2: along b = z), virtual elements
// vfirst[m] .. vfirst[m+1]-1.  Slot s: the mortar face of an element, whose FV
// neighbour values are gathered into Tables::mnb when the element is FV.
struct MortarTables {
    int n_elem;
    const int32_t* big;
    const uint8_t* fB;
    const uint8_t* split;
    const int32_t* vfirst;
    const int32_t* vmort;   // per virtual element
    const uint8_t* vquad;   // quadrant qa + 2 qb
    const int32_t* vsmall;  // the small element across
    const int32_t* selem;   // per slot: owner element
    const uint8_t* sface;   // owner's face
    const int32_t* smort;   // mortar
    const int8_t* squad;    // owner's quadrant, -1 for the big side
};

struct Buffers {
    double* fu;     // width V : DG trace of u / FV boundary sub-cell means
    double* fg;     // width 3V: DG trace of the lifted gradient / FV boundary-cell gradient
    double* flux;   // width V : outward normal flux on the element's own representation
    double* flift;  // width V : BR1 lifting value U* (DG elements)
    double* frec;   // width V : FV reconstructed state at the element face
    double* rtmp;   // state-sized: volume part (DG) / interior sub-cell part (FV) of -R
};

// Adjoint face buffers (same slot layout as the forward face buffers).
struct AdjBuffers {
    double* fbar;  // width V : adjoint of the outward face fluxes
    double* ubar;  // width V : adjoint of the face values u(+-1)
    double* gbar;  // width 3V: adjoint of the gradient traces
    double* sbar;  // width V : adjoint of the lifting values U*
};

struct Params {
    DevPhys ph;
    Tables t;
    Buffers b;
    const double* bank;
    BankIdx bi;
    int nfv;
    int* status;  // device status word (first error wins)
};

// A tile is a run of `count` items (elements or faces) of one kind and size,
// stored consecutively in `items` from `first`.
struct Tiles {
    const int32_t* first;
    const int32_t* count;
    const uint8_t* n;     // points per direction of the items (or common-representation size)
    const int32_t* items;
};

// Tiles of faces that need no change of representation: every face of a tile
// has the same direction d and the same number of points per direction nc.
struct FaceTiles {
    const int32_t* first;
    const int32_t* count;
    const uint8_t* nc;
    const uint8_t* d;
    const int32_t* items;  // face ids
};

// Faces: lower element L (across its +d face) and upper element R (its -d face).
struct Faces {
    const int32_t* L;
    const int32_t* R;
    const uint8_t* d;
};

// Shared-memory layout of one FV element in k_fv (offsets in doubles); gs = 1
// keeps the sub-cell gradients (see the kernel).
struct FvLayout {
    int u, w, nb, nw, f, g, t, total;
};

__host__ __device__ __forceinline__ FvLayout fv_layout(int V, int n, int gs) {
    // tmp: the neighbour gather's scratch, per face a layer of at most MAXP^2
    // points and its half-mapped form (n x MAXP) for all six faces at once
    // fl: the interior face fluxes of the three directions (of two with gs = 2,
    // which runs the z faces in a second pass)
    const int n2 = n * n, n3 = n2 * n, tmp = 6 * V * (MAXP * MAXP + n * MAXP),
              fl = (gs == 2 ? 2 : 3) * V * (n - 1) * n2;
    FvLayout L;
    if (gs) {
        const int gsz = 3 * V * n3 > tmp ? 3 * V * n3 : tmp;
        L.g = 0;
        L.t = 0;
        L.w = gsz;
        L.nw = L.w + V * n3;
        L.f = L.nw + 6 * V * n2;
        L.u = L.f;
        L.nb = L.f + V * n3;
        L.total = L.f + (fl > V * n3 + 6 * V * n2 ? fl : V * n3 + 6 * V * n2);
    } else {
        L.u = 0;
        L.w = V * n3;
        L.nb = 2 * V * n3;
        L.nw = L.nb + 6 * V * n2;
        L.f = L.nw + 6 * V * n2;
        L.t = L.f;
        L.g = 0;
        L.total = L.f + (fl > tmp ? fl : tmp);
    }
    return L;
}

__host__ __device__ __forceinline__ int node_index(int n, int d, int m, int a, int b) {
    return d == 0 ? m + n * (a + n * b) : (d == 1 ? a + n * (m + n * b) : a + n * (b + n * m));
}

// Non-finite test on the exponent bits (integer pipe; the FP64 pipe is the
// bottleneck of every kernel here).
__device__ __forceinline__ bool nonfinite_bits(double x) {
    return ((__double2hiint(x) >> 20) & 0x7ff) == 0x7ff;
}

// Device status word: status[0] the first error code (first error wins),
// status[1] the element it was detected in.
__device__ __forceinline__ void set_status(int* status, int code, int elem) {
    if (status && atomicCAS(status, 0, code) == 0) atomicExch(status + 1, elem);
}

}  // namespace dgfv
