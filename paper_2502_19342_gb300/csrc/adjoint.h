// Host-side launchers of the adjoint kernels in adjoint.cu.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "common.cuh"

namespace dgfv {

void launch_adj_surface(int nk, const Params& P, const AdjBuffers& A, const Tiles& T, int ntiles, const double* Rb,
                        cudaStream_t s);
// Mortars, transposed: which 0/1 = fluxes / lifting values onto the virtual
// sides (launch_adj_mortar_virt), gradient / value traces back onto the big
// side (launch_adj_mortar_big).
void launch_adj_mortar_virt(int nk, const Params& P, const AdjBuffers& A, const MortarTables& M, int n_virt,
                            int which, cudaStream_t s);
void launch_adj_mortar_big(int nk, const Params& P, const AdjBuffers& A, const MortarTables& M, int n_mort,
                           int which, cudaStream_t s);
void launch_adj_faces(int nk, const Params& P, const AdjBuffers& A, const Faces& F, const FaceTiles& conf,
                      int nconf, cudaStream_t s);
// Mixed faces in three passes on the forward's mixed-face tiles and scratch.
void launch_adj_mixed_faces(int nk, const Params& P, const AdjBuffers& A, const Faces& F, const FaceTiles& T,
                            int ntiles, const int32_t* mface, const int64_t* mpt, int nmixed, double* Sin,
                            double* Sout, cudaStream_t s);
size_t adj_volume_smem_bytes(int nk, int n, int count);
void launch_adj_vol_a(int nk, const Params& P, const Tiles& T, int ntiles, size_t smem, const double* U,
                      const double* Rb, double* Ub, double* gvol, double* gf, cudaStream_t s, int split = 0);
// Split form (Sec. 3.5): reverse of the two-point volume term, added to Ub.
size_t adj_split_smem_bytes(int nk, int n, int count);
void launch_adj_split(int nk, const Params& P, const Tiles& T, int ntiles, size_t smem, const double* U,
                      const double* Rb, double* Ub, cudaStream_t s);
void launch_adj_vol_b(int nk, const Params& P, const AdjBuffers& A, const Tiles& T, int ntiles, size_t smem,
                      const double* gvol, double* Ub, cudaStream_t s);
void launch_adj_lift(int nk, const Params& P, const AdjBuffers& A, const Faces& F, const int32_t* list, int nfaces,
                     cudaStream_t s);
// Mortar faces of FV elements: the transposes of the neighbour-value gathers.
void launch_adj_mortar_nb(int nk, const Params& P, const AdjBuffers& A, const MortarTables& M, int n_mort,
                          double* Ub, cudaStream_t s);
// FV sub-cell elements (one tile per element): the surface adjoint, then after
// the face and lifting adjoints the element reverse and the gather of the
// neighbour-layer adjoints into the neighbours' U_bar (all elements).
size_t adj_fv_smem_bytes(int nk, int nfv);
void launch_adj_surface_fv(int nk, const Params& P, const AdjBuffers& A, const Tiles& T, int ntiles, const double* Rb,
                           cudaStream_t s);
void launch_adj_fv_elements(int nk, const Params& P, const AdjBuffers& A, const Tiles& T, int ntiles,
                            const double* U, const double* Rb, double* Ub, double* gf, double* gvol, double* fvs,
                            int64_t cap_state, int n_elem, cudaStream_t s);
void launch_adj_prolong(int nk, const Params& P, const AdjBuffers& A, const Tiles& T, int ntiles, double* Ub,
                        cudaStream_t s);
void launch_axpby(int64_t n, double a, const double* x, double b, const double* y, double* out, cudaStream_t s);
// SSP-RK3 step-adjoint combinations (see k_rk3_adj_combine).
void launch_rk3_adj_combine(int64_t n, int mode, double c1, double c2, double dt, const double* x, const double* y,
                            double* o1, double* o2, cudaStream_t s);

}  // namespace dgfv
