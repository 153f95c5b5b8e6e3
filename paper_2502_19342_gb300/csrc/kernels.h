// Host-side launchers of the forward kernels (kernels.cu, fv.cu, volume.cu; no
// torch types).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "common.cuh"

namespace dgfv {

void launch_prolong(int nk, const Params& P, const Tiles& T, int ntiles, const double* U, cudaStream_t s);
size_t fv_smem_bytes(int nk, int nfv);
// faces_only: only the element-face states and boundary gradients (frec, fg),
// not the sub-cell fluxes (the adjoint's recomputation of the forward).
// variant: 0 automatic, 1 gradients recomputed at each face, 2 gradients kept
// in shared memory, 3 kept with the z faces in a second pass (when that layout
// fits).
void launch_fv(int nk, const Params& P, const Tiles& T, int ntiles, const double* U, cudaStream_t s,
               bool faces_only = false, int variant = 0);
void launch_face_lift_conf(int nk, const Params& P, const Faces& F, const FaceTiles& T, int ntiles, cudaStream_t s);
void launch_face_lift(int nk, const Params& P, const Faces& F, const int32_t* list, int nfaces, cudaStream_t s);
size_t volume_smem_bytes(int nk, int n, int count);
size_t volume_split_smem_bytes(int nk, int n, int count, bool viscous);
void launch_dg_volume_split(int nk, const Params& P, const Tiles& T, int ntiles, size_t smem, const double* U,
                            cudaStream_t s);
void launch_dg_volume(int nk, const Params& P, const Tiles& T, int ntiles, size_t smem, const double* U,
                      cudaStream_t s, int variant = 0);
// Persistent form (one launch over every degree, min(ntiles, resident CTAs)
// CTAs taking tiles from the counter `queue`, which the launch zeroes).
void launch_dg_volume_persistent(int nk, const Params& P, const Tiles& T, int ntiles, size_t smem, const double* U,
                                 cudaStream_t s, int variant, int* queue, int n_sm);
void launch_mixed_faces(int nk, const Params& P, const Faces& F, const FaceTiles& T, int ntiles, const int32_t* mface,
                        const int64_t* mpt, int nmixed, double* Sin, double* Sout, cudaStream_t s);
void launch_face_flux_conf(int nk, const Params& P, const Faces& F, const FaceTiles& T, int ntiles, cudaStream_t s);
// Mortars (Sec. 3.2.3): virtual small sides from the big side (pass 0: u /
// FV state and gradient, pass 1: DG gradient), projection back (which 0:
// lifting values, 1: fluxes), FV neighbour values of mortar faces.
void launch_mortar_in(int nk, const Params& P, const MortarTables& M, int n_virt, int pass, cudaStream_t s);
void launch_mortar_out(int nk, const Params& P, const MortarTables& M, int n_mort, int which, cudaStream_t s);
void launch_mortar_nb(int nk, const Params& P, const MortarTables& M, const int32_t* active, int n_active,
                      const double* U, double* out, cudaStream_t s);
void launch_surface(int nk, const Params& P, const Tiles& T, int ntiles, const double* Uin, const double* U0,
                    double* out, int mode, double a, double b, const double* dt, bool fuse, double* dU,
                    cudaStream_t s);
void launch_dt(int nk, const Params& P, const Tiles& T, int ntiles, const double* U, double cfl_c, double cfl_v,
               double* partial, double* out3, cudaStream_t s);
void launch_pp_limit(int nk, const Params& P, const int32_t* items, int n_dg, double* U, double eps,
                     unsigned long long* count, bool write_faces, cudaStream_t s);
void launch_set_scalar(double* p, double v, cudaStream_t s);
// n doubles from src to dst by a grid-stride kernel on every SM (device
// memory, or page-locked host memory through its device mapping).
void launch_copy_state(double* dst, const double* src, int64_t n, int n_sm, cudaStream_t s);
// Time step with the per-block minima in a fixed device array (no allocation).
// Returns 0, 1 when ntiles exceeds DT_NOALLOC_MAX_BLOCKS, 2 on a CUDA error.
constexpr int DT_NOALLOC_MAX_BLOCKS = 65536;
constexpr int DT_NOALLOC_MAX_DEVICES = 64;
int launch_dt_noalloc(int nk, const Params& P, const Tiles& T, int ntiles, const double* U, double cfl_c,
                      double cfl_v, double* out3, cudaStream_t s);
void launch_indicator(int nk, const Params& P, const double* U, int n_elem, double* Ip, double* Ih, uint8_t* dec,
                      const double thr[4], int N_min, int N_max, int vars, cudaStream_t s);
void launch_remap(const Params& P, const uint8_t* n_old, const uint8_t* N_old, const uint8_t* fv_old,
                  const int64_t* off_old, const uint8_t* n_new, const uint8_t* N_new, const uint8_t* fv_new,
                  const int64_t* off_new, int V, int n_elem, const double* Uo, double* Un, int nmax,
                  cudaStream_t s);
double probe_dfma(int iters, cudaStream_t s);
double probe_dmma(int iters, cudaStream_t s);

}  // namespace dgfv
