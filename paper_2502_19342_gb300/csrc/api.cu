// C ABI of the dgfv library (include/dgfv.h): context, mesh tables, element
// layout, work tiles, face lists, stage sequencing and CUDA-graph replay.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/dgfv.h"
#include "adjoint.h"
#include "bank.h"
#include "common.cuh"
#include "kernels.h"

using namespace dgfv;

namespace {

// A named range on the host timeline of a profiler attached through NVTX
// (header-only NVTX 3; without a tool the push and pop return at once).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

struct TileSet {
    std::vector<int32_t> first, count, items;
    std::vector<uint8_t> n;
    std::vector<int> bin_first, bin_count;  // consecutive tiles of one point count
    std::vector<size_t> bin_smem;
    int32_t *d_first = nullptr, *d_count = nullptr, *d_items = nullptr;
    uint8_t* d_n = nullptr;
    int ntiles = 0;
    size_t smem = 0;
    Tiles view() const { return Tiles{d_first, d_count, d_n, d_items}; }
    Tiles view(int tile0) const { return Tiles{d_first + tile0, d_count + tile0, d_n + tile0, d_items}; }
};

struct FaceList {
    std::vector<int32_t> ids;
    int32_t* d = nullptr;
    int count = 0;
};

struct FaceTileSet {
    std::vector<int32_t> first, count, items;
    std::vector<uint8_t> nc, d;
    std::vector<int> bin_first, bin_count;  // consecutive tiles of one (direction, point count)
    int32_t *d_first = nullptr, *d_count = nullptr, *d_items = nullptr;
    uint8_t *d_nc = nullptr, *d_d = nullptr;
    int ntiles = 0;
    FaceTiles view() const { return FaceTiles{d_first, d_count, d_nc, d_d, d_items}; }
    FaceTiles view(int t0) const { return FaceTiles{d_first + t0, d_count + t0, d_nc + t0, d_d + t0, d_items}; }
};

// Faces that change representation, grouped like the conforming tiles by
// (direction, common point count); face[k], pt[k] (scratch point offset) per
// mixed face k in tile order.
struct MixedSet {
    FaceTileSet tiles;
    std::vector<int32_t> face;
    std::vector<int64_t> pt;
    int32_t* d_face = nullptr;
    int64_t* d_pt = nullptr;
    int n = 0;
    int64_t cap_pts = 0;              // capacity of the scratch in face points
    double *d_in = nullptr, *d_out = nullptr;  // 4V and V values per point
};

enum Kernel { K_PROLONG = 0, K_FV, K_LIFT, K_VOLUME, K_FLUX, K_SURFACE, K_DT, K_INDICATOR, K_REMAP, K_COUNT };

struct Profiler {
    bool on = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[K_COUNT];
    size_t used[K_COUNT] = {};
};

}  // namespace

struct dgfv_ctx {
    int dev = 0;
    int nk = 2, V = 6;
    DevPhys ph{};
    dgfv_opts opts{};
    int N_min = 1, N_max = 1, nfv = 2;
    bool fv_own = false;  // per-element sub-cell counts: an FV element of degree N has N+1
    int n_elem = 0, n_faces = 0;
    std::vector<int32_t> nb;
    std::vector<double> rh;
    std::vector<int32_t> faceL, faceR;
    std::vector<uint8_t> faceD;
    // current pattern and layout
    std::vector<uint8_t> N, fv, npts;
    std::vector<int64_t> off, fo;
    int64_t n_state = 0, n_fpts = 0;
    int64_t cap_state = 0, cap_fpts = 0;
    // device tables (current and previous pattern, for the remap)
    uint8_t *d_n = nullptr, *d_N = nullptr, *d_fv = nullptr;
    int64_t *d_off = nullptr, *d_fo = nullptr;
    uint8_t *d_n_old = nullptr, *d_N_old = nullptr, *d_fv_old = nullptr;
    int64_t* d_off_old = nullptr;
    int32_t* d_nb = nullptr;
    double* d_rh = nullptr;
    int32_t *d_faceL = nullptr, *d_faceR = nullptr;
    uint8_t* d_faceD = nullptr;
    double* d_bank = nullptr;
    BankIdx bi{};
    // buffers
    double *d_fu = nullptr, *d_fg = nullptr, *d_flux = nullptr, *d_flift = nullptr, *d_frec = nullptr;
    double *d_rtmp = nullptr, *d_U = nullptr, *d_Us = nullptr;
    double *d_dt3 = nullptr, *d_partial = nullptr;
    double *d_Ip = nullptr, *d_Ih = nullptr;
    uint8_t* d_dec = nullptr;
    int* d_status = nullptr;
    unsigned long long* d_pp_count = nullptr;  // elements changed by the stage limiter
    TileSet all, dg, fvt;
    FaceList lift, flux;    // flux: faces that change representation
    FaceTileSet conf;       // faces with one representation on both sides
    MixedSet mixed;         // the flux faces in three passes
    int n_fv_elems = 0;
    int launch_mode = 0;           // 0: one launch per kernel; 1: one launch per degree bin;
                                   // 2: as 0 with the volume kernel persistent (work queue)
    int* d_queue = nullptr;        // work-queue counter of the persistent volume kernel
    int n_sm = 1;                  // SMs of the context's device
    int fv_variant = 0;            // k_fv layout: 0 automatic, 1 gradients recomputed, 2 kept, 3 kept + two face passes
    int vol_per_tile[MAXDG + 1] = {};  // elements per volume tile (0: default), set by the autotuner
    int vol_variant = 0;              // volume-kernel launch variant (threads, register budget), autotuned
    bool state_valid = false;
    std::string err;
    // graph of one RK step
    cudaGraphExec_t graph = nullptr;
    bool graph_valid = false;
    double graph_dt = 0.0;
    cudaStream_t graph_stream = nullptr;
    Profiler prof;
    // non-conforming interfaces (Sec. 3.2.3); virtual element v is entry n_elem + v
    int n_mort = 0, n_virt = 0, n_slot = 0, n_slot_active = 0;
    std::vector<int32_t> m_big, m_vfirst, v_mort, v_small, s_elem, s_mort, s_nbe;
    std::vector<uint8_t> m_fB, m_split, v_quad, s_face;
    std::vector<int8_t> s_quad;
    int32_t *d_m_big = nullptr, *d_m_vfirst = nullptr, *d_v_mort = nullptr, *d_v_small = nullptr;
    int32_t *d_s_elem = nullptr, *d_s_mort = nullptr, *d_s_nbe = nullptr, *d_s_active = nullptr;
    uint8_t *d_m_fB = nullptr, *d_m_split = nullptr, *d_v_quad = nullptr, *d_s_face = nullptr;
    int8_t* d_s_quad = nullptr;
    double* d_mnb = nullptr;  // FV neighbour values per slot, V x N_FV^2
    // adjoint buffers, allocated by the first adjoint call
    bool adj_ready = false;
    double *d_fbar = nullptr, *d_ubar = nullptr, *d_gbar = nullptr, *d_sbar = nullptr;
    double *d_S1 = nullptr, *d_S2 = nullptr, *d_B1 = nullptr, *d_B2 = nullptr, *d_W = nullptr;
    double* d_gvol = nullptr;  // nodal gradient adjoint, 3 x state
    double* d_gf = nullptr;    // lifted gradient and volume-flux adjoint per node, 6 x state
    double* d_fvs = nullptr;   // FV element adjoint scratch (reconstruction-variable and direct adjoints), 2 x state
    size_t adj_smem = 0, adj_split_smem = 0;
    std::vector<void*> allocs;
};

namespace {

int fail(dgfv_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return fail(c, DGFV_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

template <class T>
int dalloc(dgfv_ctx* c, T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return fail(c, DGFV_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    c->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return DGFV_OK;
}

#define TRY(x)                 \
    do {                       \
        int r_ = (x);          \
        if (r_ != DGFV_OK) return r_; \
    } while (0)

Params params(const dgfv_ctx* c) {
    Params P{};
    P.ph = c->ph;
    P.t = Tables{c->d_n, c->d_N, c->d_fv, c->d_off, c->d_fo, c->d_nb, c->d_rh, c->d_mnb, c->d_s_nbe};
    P.b = Buffers{c->d_fu, c->d_fg, c->d_flux, c->d_flift, c->d_frec, c->d_rtmp};
    P.bank = c->d_bank;
    P.bi = c->bi;
    P.nfv = c->nfv;
    P.status = c->d_status;
    return P;
}

MortarTables mortar_tables(const dgfv_ctx* c) {
    return MortarTables{c->n_elem,    c->d_m_big,  c->d_m_fB,   c->d_m_split, c->d_m_vfirst, c->d_v_mort,
                        c->d_v_quad,  c->d_v_small, c->d_s_elem, c->d_s_face,  c->d_s_mort,   c->d_s_quad};
}

// Brackets one kernel launch with events when profiling is on.
struct Timed {
    dgfv_ctx* c;
    int k;
    cudaStream_t s;
    Timed(dgfv_ctx* c_, int k_, cudaStream_t s_) : c(c_), k(k_), s(s_) {
        if (!c->prof.on) return;
        auto& pool = c->prof.ev[k];
        if (c->prof.used[k] == pool.size()) {
            cudaEvent_t a, b;
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            pool.emplace_back(a, b);
        }
        cudaEventRecord(pool[c->prof.used[k]].first, s);
    }
    ~Timed() {
        if (!c->prof.on) return;
        cudaEventRecord(c->prof.ev[k][c->prof.used[k]].second, s);
        c->prof.used[k]++;
    }
};

int build_bank(dgfv_ctx* c) {
    std::vector<double> bank;
    auto put = [&](const std::vector<double>& v) {
        const int32_t o = (int32_t)bank.size();
        bank.insert(bank.end(), v.begin(), v.end());
        return o;
    };
    std::memset(&c->bi, 0, sizeof(c->bi));
    const int kind = c->opts.nodes;
    for (int n = c->N_min + 1; n <= c->N_max + 1; ++n) {
        Bank1D b = make_bank(n, kind);
        c->bi.dhat[n] = put(b.Dhat);
        c->bi.w[n] = put(b.w);
        if (c->opts.split_form) {
            // 2D - W^{-1}B: the boundary correction -(B_ii/w_i) F(u_i) folded into the diagonal
            std::vector<double> S(n * n);
            for (int i = 0; i < n * n; ++i) S[i] = 2.0 * b.D[i];
            S[0] += 1.0 / b.w[0];
            S[n * n - 1] -= 1.0 / b.w[n - 1];
            c->bi.dsplit[n] = put(S);
        }
        c->bi.lm[n] = put(b.lm);
        c->bi.lp[n] = put(b.lp);
        c->bi.lhm[n] = put(b.lhm);
        c->bi.lhp[n] = put(b.lhp);
        c->bi.vinv[n] = put(b.vinv);
        // V^{DG->FV} / V^{FV->DG} to the global sub-cell count, or (per-element
        // counts) to every count an FV element can have
        for (int m = c->fv_own ? c->N_min + 1 : c->nfv; m <= (c->fv_own ? c->N_max + 1 : c->nfv); ++m) {
            c->bi.d2f[n][m] = put(make_dg2fv(n, m, kind));
            c->bi.f2d[n][m] = put(m >= n ? make_fv2dg(n, m, kind) : make_fv2dg_l2(n, m, kind));
            if (c->fv_own) c->bi.ov[n][m] = put(make_fv_overlap(n, m));
        }
        for (int m = c->N_min + 1; m <= c->N_max + 1; ++m) c->bi.vm[n][m] = put(make_vmap(n, m, kind));
        for (int h = 0; h < 2; ++h) {
            c->bi.mi[n][h] = put(make_mortar(n, h, false, kind));
            c->bi.mp[n][h] = put(make_mortar(n, h, true, kind));
        }
    }
    for (int h = 0; h < 2; ++h) {
        c->bi.mfi[h] = put(make_mortar_fv(c->nfv, h, false));
        c->bi.mfp[h] = put(make_mortar_fv(c->nfv, h, true));
    }
    for (int n = 1; n <= MAXP; ++n) {
        std::vector<double> I((size_t)n * n, 0.0);
        for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = 1.0;
        c->bi.eye[n] = put(I);
    }
    TRY(dalloc(c, &c->d_bank, bank.size()));
    CK(cudaMemcpy(c->d_bank, bank.data(), bank.size() * sizeof(double), cudaMemcpyHostToDevice));
    return DGFV_OK;
}

int upload_tiles(dgfv_ctx* c, TileSet& t) {
    t.ntiles = (int)t.first.size();
    if (t.ntiles == 0) return DGFV_OK;
    CK(cudaMemcpy(t.d_first, t.first.data(), t.ntiles * sizeof(int32_t), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(t.d_count, t.count.data(), t.ntiles * sizeof(int32_t), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(t.d_n, t.n.data(), t.ntiles * sizeof(uint8_t), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(t.d_items, t.items.data(), t.items.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    return DGFV_OK;
}

// Group items by their point count n and cut each group into tiles of at most
// per_tile(n) items.  The groups go in descending n: the block scheduler
// dispatches tiles in order, so the heaviest tiles start first and the light
// ones fill the tail of a mixed-degree launch (longest first).
template <class Sel, class Per>
void make_tiles(const dgfv_ctx* c, TileSet& t, Sel sel, Per per_tile) {
    t.first.clear(); t.count.clear(); t.items.clear(); t.n.clear();
    t.bin_first.clear(); t.bin_count.clear();
    for (int n = MAXP; n >= 1; --n) {
        std::vector<int32_t> group;
        for (int e = 0; e < c->n_elem; ++e)
            if (c->npts[e] == n && sel(e)) group.push_back(e);
        if (group.empty()) continue;
        const int per = std::max(1, per_tile(n));
        t.bin_first.push_back((int)t.first.size());
        t.bin_count.push_back((int)((group.size() + per - 1) / per));
        for (size_t s = 0; s < group.size(); s += per) {
            const int cnt = (int)std::min<size_t>(per, group.size() - s);
            t.first.push_back((int32_t)t.items.size());
            t.count.push_back(cnt);
            t.n.push_back((uint8_t)n);
            t.items.insert(t.items.end(), group.begin() + s, group.begin() + s + cnt);
        }
    }
}

// Shared memory of one volume tile (standard or split form).
size_t vol_smem(const dgfv_ctx* c, int n, int count) {
    return c->opts.split_form ? volume_split_smem_bytes(c->nk, n, count, c->ph.viscous != 0)
                              : volume_smem_bytes(c->nk, n, count);
}

// The volume kernel of the context's scheme.
void launch_volume(const dgfv_ctx* c, const Params& P, const Tiles& T, int ntiles, size_t smem, const double* U,
                   cudaStream_t s, int variant) {
    if (c->opts.split_form)
        launch_dg_volume_split(c->nk, P, T, ntiles, smem, U, s);
    else
        launch_dg_volume(c->nk, P, T, ntiles, smem, U, s, variant);
}

// Elements per volume tile: about 256 nodes per CTA unless autotuned.
int volume_per_tile(const dgfv_ctx* c, int n) {
    return c->vol_per_tile[n] > 0 ? c->vol_per_tile[n] : std::max(1, 256 / (n * n * n));
}

int apply_layout(dgfv_ctx* c) {
    const int ne = c->n_elem, nt = ne + c->n_virt;
    c->npts.resize(nt);
    c->off.resize(ne);
    c->fo.resize(nt);
    c->N.resize(nt);
    c->fv.resize(nt);
    int64_t so = 0, fpo = 0;
    c->n_fv_elems = 0;
    for (int e = 0; e < ne; ++e) {
        const int n = (c->fv[e] && !c->fv_own) ? c->nfv : c->N[e] + 1;
        c->npts[e] = (uint8_t)n;
        c->off[e] = so;
        c->fo[e] = fpo;
        so += (int64_t)c->V * n * n * n;
        fpo += 6LL * n * n;
        c->n_fv_elems += c->fv[e] ? 1 : 0;
    }
    // virtual small sides take the representation of their big element; they
    // use face slots 0 and 1 only
    for (int v = 0; v < c->n_virt; ++v) {
        const int eb = c->m_big[c->v_mort[v]], e = ne + v;
        c->N[e] = c->N[eb];
        c->fv[e] = c->fv[eb];
        c->npts[e] = c->npts[eb];
        c->fo[e] = fpo;
        fpo += 2LL * c->npts[e] * c->npts[e];
    }
    c->n_state = so;
    c->n_fpts = fpo;
    CK(cudaMemcpy(c->d_n, c->npts.data(), nt, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_N, c->N.data(), nt, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_fv, c->fv.data(), nt, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_off, c->off.data(), ne * sizeof(int64_t), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_fo, c->fo.data(), nt * sizeof(int64_t), cudaMemcpyHostToDevice));
    // mortar faces of FV elements need their neighbour values gathered
    {
        std::vector<int32_t> act;
        for (int sl = 0; sl < c->n_slot; ++sl)
            if (c->fv[c->s_elem[sl]]) act.push_back(sl);
        c->n_slot_active = (int)act.size();
        if (!act.empty())
            CK(cudaMemcpy(c->d_s_active, act.data(), act.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    // tiles
    make_tiles(c, c->all, [](int) { return true; }, [](int n) { return std::max(1, 512 / (n * n * n)); });
    make_tiles(c, c->dg, [&](int e) { return !c->fv[e]; }, [&](int n) { return volume_per_tile(c, n); });
    make_tiles(c, c->fvt, [&](int e) { return c->fv[e] != 0; }, [](int) { return 1; });
    size_t sm = 0;
    c->dg.bin_smem.assign(c->dg.bin_first.size(), 0);
    for (size_t b = 0; b < c->dg.bin_first.size(); ++b)
        for (int t = c->dg.bin_first[b]; t < c->dg.bin_first[b] + c->dg.bin_count[b]; ++t) {
            const size_t x = vol_smem(c, c->dg.n[t], c->dg.count[t]);
            c->dg.bin_smem[b] = std::max(c->dg.bin_smem[b], x);
            sm = std::max(sm, x);
        }
    c->dg.smem = sm;
    size_t asm_ = 0;
    size_t ssm = 0;
    for (int t = 0; t < (int)c->dg.first.size(); ++t) {
        asm_ = std::max(asm_, adj_volume_smem_bytes(c->nk, c->dg.n[t], c->dg.count[t]));
        ssm = std::max(ssm, adj_split_smem_bytes(c->nk, c->dg.n[t], c->dg.count[t]));
    }
    c->adj_smem = asm_;
    c->adj_split_smem = ssm;
    TRY(upload_tiles(c, c->all));
    TRY(upload_tiles(c, c->dg));
    TRY(upload_tiles(c, c->fvt));
    // face lists: lifting needs a DG side; the flux of a face whose sides share
    // one representation runs in the conforming kernel, the rest in the mixed one
    c->lift.ids.clear();
    c->flux.ids.clear();
    std::vector<int32_t> conf_by[3][MAXP + 1];
    for (int f = 0; f < c->n_faces; ++f) {
        const int L = c->faceL[f], R = c->faceR[f];
        const bool same = c->fv[L] == c->fv[R] && c->npts[L] == c->npts[R];
        if (same)
            conf_by[c->faceD[f]][c->npts[L]].push_back(f);
        else
            c->flux.ids.push_back(f);
        if (!(c->fv[L] && c->fv[R])) c->lift.ids.push_back(f);
    }
    {
        FaceTileSet& t = c->conf;
        t.first.clear(); t.count.clear(); t.items.clear(); t.nc.clear(); t.d.clear();
        t.bin_first.clear(); t.bin_count.clear();
        for (int d = 0; d < 3; ++d)
            for (int n = MAXP; n >= 1; --n) {  // descending, as the element tiles
                const auto& g = conf_by[d][n];
                const int per = std::max(1, 256 / (n * n));
                if (!g.empty()) {
                    t.bin_first.push_back((int)t.first.size());
                    t.bin_count.push_back((int)((g.size() + per - 1) / per));
                }
                for (size_t s0 = 0; s0 < g.size(); s0 += per) {
                    const int cnt = (int)std::min<size_t>(per, g.size() - s0);
                    t.first.push_back((int32_t)t.items.size());
                    t.count.push_back(cnt);
                    t.nc.push_back((uint8_t)n);
                    t.d.push_back((uint8_t)d);
                    t.items.insert(t.items.end(), g.begin() + s0, g.begin() + s0 + cnt);
                }
            }
        t.ntiles = (int)t.first.size();
        if (t.ntiles) {
            CK(cudaMemcpy(t.d_first, t.first.data(), t.ntiles * sizeof(int32_t), cudaMemcpyHostToDevice));
            CK(cudaMemcpy(t.d_count, t.count.data(), t.ntiles * sizeof(int32_t), cudaMemcpyHostToDevice));
            CK(cudaMemcpy(t.d_nc, t.nc.data(), t.ntiles, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(t.d_d, t.d.data(), t.ntiles, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(t.d_items, t.items.data(), t.items.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
        }
    }
    {
        // mixed faces: common representation N_FV sub-cells or the higher degree
        MixedSet& m = c->mixed;
        FaceTileSet& t = m.tiles;
        t.first.clear(); t.count.clear(); t.items.clear(); t.nc.clear(); t.d.clear();
        m.face.clear();
        m.pt.clear();
        std::vector<int32_t> by[3][MAXP + 1];
        for (int32_t f : c->flux.ids) {
            const int L = c->faceL[f], R = c->faceR[f];
            // as mixed_face: DG/FV on the FV side's sub-cells, else the larger count
            const int nc = (c->fv[L] != c->fv[R]) ? (c->fv[L] ? c->npts[L] : c->npts[R])
                                                  : std::max<int>(c->npts[L], c->npts[R]);
            by[c->faceD[f]][nc].push_back(f);
        }
        int64_t pts = 0;
        for (int d = 0; d < 3; ++d)
            for (int nc = 1; nc <= MAXP; ++nc) {
                const auto& g = by[d][nc];
                const int per = std::max(1, 128 / (nc * nc));
                for (size_t s0 = 0; s0 < g.size(); s0 += per) {
                    const int cnt = (int)std::min<size_t>(per, g.size() - s0);
                    t.first.push_back((int32_t)t.items.size());
                    t.count.push_back(cnt);
                    t.nc.push_back((uint8_t)nc);
                    t.d.push_back((uint8_t)d);
                    for (int q = 0; q < cnt; ++q) {
                        t.items.push_back((int32_t)m.face.size());
                        m.face.push_back(g[s0 + q]);
                        m.pt.push_back(pts);
                        pts += nc * nc;
                    }
                }
            }
        t.ntiles = (int)t.first.size();
        m.n = (int)m.face.size();
        if (pts > m.cap_pts) {  // grow the scratch (graphs are recaptured after a layout change)
            for (double** q : {&m.d_in, &m.d_out}) {
                if (*q) {
                    cudaFree(*q);
                    c->allocs.erase(std::find(c->allocs.begin(), c->allocs.end(), (void*)*q));
                    *q = nullptr;
                }
            }
            m.cap_pts = pts + pts / 4;
            TRY(dalloc(c, &m.d_in, (size_t)m.cap_pts * 4 * c->V));
            TRY(dalloc(c, &m.d_out, (size_t)m.cap_pts * c->V));
        }
        if (t.ntiles) {
            CK(cudaMemcpy(t.d_first, t.first.data(), t.ntiles * sizeof(int32_t), cudaMemcpyHostToDevice));
            CK(cudaMemcpy(t.d_count, t.count.data(), t.ntiles * sizeof(int32_t), cudaMemcpyHostToDevice));
            CK(cudaMemcpy(t.d_nc, t.nc.data(), t.ntiles, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(t.d_d, t.d.data(), t.ntiles, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(t.d_items, t.items.data(), t.items.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
            CK(cudaMemcpy(m.d_face, m.face.data(), m.n * sizeof(int32_t), cudaMemcpyHostToDevice));
            CK(cudaMemcpy(m.d_pt, m.pt.data(), m.n * sizeof(int64_t), cudaMemcpyHostToDevice));
        }
    }
    c->lift.count = (int)c->lift.ids.size();
    c->flux.count = (int)c->flux.ids.size();
    if (c->lift.count)
        CK(cudaMemcpy(c->lift.d, c->lift.ids.data(), c->lift.count * sizeof(int32_t), cudaMemcpyHostToDevice));
    if (c->flux.count)
        CK(cudaMemcpy(c->flux.d, c->flux.ids.data(), c->flux.count * sizeof(int32_t), cudaMemcpyHostToDevice));
    c->graph_valid = false;
    return DGFV_OK;
}

int alloc_tiles(dgfv_ctx* c, TileSet& t) {
    TRY(dalloc(c, &t.d_first, c->n_elem));
    TRY(dalloc(c, &t.d_count, c->n_elem));
    TRY(dalloc(c, &t.d_n, c->n_elem));
    TRY(dalloc(c, &t.d_items, c->n_elem));
    return DGFV_OK;
}

// One evaluation of R on Uin; the surface kernel writes mode 0: out = R, or
// mode 1: out = a*U0 + b*(Uin + dt*R).
// One evaluation of R(Uin) and, in mode 1 (SSP-RK3) or 2 (low-storage RK4,
// dU in d_Us, out = Uin), the stage update.  have_faces:
// the face values of Uin are already in the face buffer (written by the
// previous stage's fused surface pass).  fuse_faces (mode 1): write the face
// values of out for the next stage.
void enqueue_stage(dgfv_ctx* c, const double* Uin, const double* U0, double* out, int mode, double a, double b,
                   cudaStream_t s, bool have_faces = false, bool fuse_faces = false) {
    const Params P = params(c);
    const Faces F{c->d_faceL, c->d_faceR, c->d_faceD};
    const bool per_bin = c->launch_mode == 1;
    double* dU = mode == 2 ? c->d_Us : nullptr;  // low-storage RK4 register
    const int n_dg = (int)c->dg.items.size();
    if (!have_faces) {
        Timed t(c, K_PROLONG, s);
        if (per_bin)
            for (size_t bi = 0; bi < c->all.bin_first.size(); ++bi)
                launch_prolong(c->nk, P, c->all.view(c->all.bin_first[bi]), c->all.bin_count[bi], Uin, s);
        else
            launch_prolong(c->nk, P, c->all.view(), c->all.ntiles, Uin, s);
    }
    const MortarTables MT = mortar_tables(c);
    if (c->n_fv_elems) {
        Timed t(c, K_FV, s);
        launch_mortar_nb(c->nk, P, MT, c->d_s_active, c->n_slot_active, Uin, c->d_mnb, s);
        launch_fv(c->nk, P, c->fvt.view(), c->fvt.ntiles, Uin, s, false, c->fv_variant);
    }
    if (c->n_mort) { Timed t(c, K_LIFT, s); launch_mortar_in(c->nk, P, MT, c->n_virt, 0, s); }
    if (c->ph.viscous) {
        // conforming DG faces one thread per point; faces that change degree or
        // type (all with a DG side) one CTA each
        Timed t(c, K_LIFT, s);
        launch_face_lift_conf(c->nk, P, F, c->conf.view(), c->conf.ntiles, s);
        launch_face_lift(c->nk, P, F, c->flux.d, c->flux.count, s);
        launch_mortar_out(c->nk, P, MT, c->n_mort, 0, s);
    }
    if (c->dg.ntiles) {
        Timed t(c, K_VOLUME, s);
        if (per_bin)
            for (size_t bi = 0; bi < c->dg.bin_first.size(); ++bi)
                launch_volume(c, P, c->dg.view(c->dg.bin_first[bi]), c->dg.bin_count[bi], c->dg.bin_smem[bi], Uin, s,
                              c->vol_variant);
        else if (c->launch_mode == 2 && !c->opts.split_form)
            launch_dg_volume_persistent(c->nk, P, c->dg.view(), c->dg.ntiles, c->dg.smem, Uin, s, c->vol_variant,
                                        c->d_queue, c->n_sm);
        else
            launch_volume(c, P, c->dg.view(), c->dg.ntiles, c->dg.smem, Uin, s, c->vol_variant);
    }
    {
        Timed t(c, K_FLUX, s);
        if (c->n_mort && c->ph.viscous) launch_mortar_in(c->nk, P, MT, c->n_virt, 1, s);
        if (per_bin)
            for (size_t bi = 0; bi < c->conf.bin_first.size(); ++bi)
                launch_face_flux_conf(c->nk, P, F, c->conf.view(c->conf.bin_first[bi]), c->conf.bin_count[bi], s);
        else
            launch_face_flux_conf(c->nk, P, F, c->conf.view(), c->conf.ntiles, s);
        launch_mixed_faces(c->nk, P, F, c->mixed.tiles.view(), c->mixed.tiles.ntiles, c->mixed.d_face, c->mixed.d_pt,
                           c->mixed.n, c->mixed.d_in, c->mixed.d_out, s);
        launch_mortar_out(c->nk, P, MT, c->n_mort, 1, s);
    }
    {
        Timed t(c, K_SURFACE, s);
        if (per_bin)
            for (size_t bi = 0; bi < c->all.bin_first.size(); ++bi)
                launch_surface(c->nk, P, c->all.view(c->all.bin_first[bi]), c->all.bin_count[bi], Uin, U0, out, mode,
                               a, b, c->d_dt3, fuse_faces, dU, s);
        else
            launch_surface(c->nk, P, c->all.view(), c->all.ntiles, Uin, U0, out, mode, a, b, c->d_dt3, fuse_faces, dU,
                           s);
    }
    if (mode != 0 && c->opts.pp_limiter && n_dg > 0) {
        // positivity limiter on the new stage state; changed elements also
        // rewrite the face values fused above
        Timed t(c, K_SURFACE, s);
        launch_pp_limit(c->nk, P, c->dg.d_items, n_dg, out, c->opts.pp_eps, c->d_pp_count, fuse_faces, s);
    }
}

// Five-stage fourth-order 2N-storage scheme (Carpenter and Kennedy), Sec. 3.3:
// dU <- A_s dU + dt R(U); U <- U + B_s dU, s = 1..5, A_1 = 0.
const double LSRK4_A[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                           -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double LSRK4_B[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                           1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                           2277821191437.0 / 14882151754819.0};

void enqueue_rk_step(dgfv_ctx* c, double dt, cudaStream_t s) {
    const Params P = params(c);
    if (dt > 0.0) {
        launch_set_scalar(c->d_dt3, dt, s);
    } else {
        Timed t(c, K_DT, s);
        launch_dt(c->nk, P, c->all.view(), c->all.ntiles, c->d_U, c->opts.cfl_c, c->opts.cfl_v, c->d_partial,
                  c->d_dt3, s);
    }
    // SSP-RK3 (Shu-Osher): U1 = U + dt R(U); U2 = 3/4 U + 1/4 (U1 + dt R(U1));
    // U <- 1/3 U + 2/3 (U2 + dt R(U2)).
    if (c->opts.integrator == DGFV_INTEGRATOR_LSRK4) {
        for (int st = 0; st < 5; ++st)
            enqueue_stage(c, c->d_U, c->d_U, c->d_U, 2, LSRK4_A[st], LSRK4_B[st], s, st > 0, st < 4);
        return;
    }
    enqueue_stage(c, c->d_U, c->d_U, c->d_Us, 1, 0.0, 1.0, s, false, true);
    enqueue_stage(c, c->d_Us, c->d_U, c->d_Us, 1, 0.75, 0.25, s, true, true);
    enqueue_stage(c, c->d_Us, c->d_U, c->d_U, 1, 1.0 / 3.0, 2.0 / 3.0, s, true, false);
}

int set_pattern(dgfv_ctx* c, const int8_t* N, const uint8_t* fv, bool remap, cudaStream_t s) {
    for (int e = 0; e < c->n_elem; ++e) {
        if (N[e] < c->N_min || N[e] > c->N_max)
            return fail(c, DGFV_ERR_ARG, "degree out of [N_min, N_max] at element " + std::to_string(e));
    }
    if (remap && c->state_valid) {
        CK(cudaMemcpyAsync(c->d_n_old, c->d_n, c->n_elem, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(c->d_N_old, c->d_N, c->n_elem, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(c->d_fv_old, c->d_fv, c->n_elem, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(c->d_off_old, c->d_off, c->n_elem * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
        CK(cudaStreamSynchronize(s));
    }
    for (int e = 0; e < c->n_elem; ++e) {
        c->N[e] = (uint8_t)N[e];
        c->fv[e] = fv ? (fv[e] ? 1 : 0) : 0;
    }
    TRY(apply_layout(c));
    if (remap && c->state_valid) {
        const Params P = params(c);
        Timed t(c, K_REMAP, s);
        launch_remap(P, c->d_n_old, c->d_N_old, c->d_fv_old, c->d_off_old, c->d_n, c->d_N, c->d_fv, c->d_off, c->V,
                     c->n_elem, c->d_U, c->d_Us,
                     std::max(c->N_max + 1, c->nfv), s);
        CK(cudaGetLastError());
        std::swap(c->d_U, c->d_Us);
        CK(cudaStreamSynchronize(s));
    } else {
        c->state_valid = false;
    }
    return DGFV_OK;
}

// Every device buffer of a context lives on the device that was current in
// dgfv_init_mesh; a call made while another device is current would launch
// there on foreign pointers, so it is refused before any CUDA work.
int check_dev(dgfv_ctx* c) {
    int d = -1;
    if (cudaGetDevice(&d) != cudaSuccess) return fail(c, DGFV_ERR_CUDA, "cudaGetDevice failed");
    if (d != c->dev)
        return fail(c, DGFV_ERR_ARG, "the current device (" + std::to_string(d) + ") is not the context's device (" +
                                         std::to_string(c->dev) + ")");
    return DGFV_OK;
}

int read_status(dgfv_ctx* c, cudaStream_t s) {
    int st[2] = {0, 0};
    CK(cudaMemcpyAsync(st, c->d_status, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (st[0] != 0) {
        const int zero[2] = {0, 0};
        CK(cudaMemcpyAsync(c->d_status, zero, 2 * sizeof(int), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
        return fail(c, st[0], std::string("device reported: ") + dgfv_status_string(st[0]) + " (element " +
                                  std::to_string(st[1]) + ")");
    }
    return DGFV_OK;
}

}  // namespace

// =============================================================================== C ABI
extern "C" {

const char* dgfv_status_string(int s) {
    switch (s) {
        case DGFV_OK: return "ok";
        case DGFV_ERR_ARG: return "invalid argument";
        case DGFV_ERR_CUDA: return "CUDA error";
        case DGFV_ERR_OOM: return "out of device memory";
        case DGFV_ERR_NONPHYSICAL: return "non-physical state (density or pressure <= 0)";
        case DGFV_ERR_NONFINITE: return "non-finite value in the state";
        case DGFV_ERR_TIMEOUT: return "bounded device wait timed out";
        case DGFV_ERR_STATE: return "call out of order";
        default: return "unknown status";
    }
}

const char* dgfv_last_error(const dgfv_ctx* c) { return c ? c->err.c_str() : "null context"; }

void dgfv_destroy(dgfv_ctx* c) {
    if (!c) return;
    if (c->graph) cudaGraphExecDestroy(c->graph);
    for (int k = 0; k < K_COUNT; ++k)
        for (auto& e : c->prof.ev[k]) {
            cudaEventDestroy(e.first);
            cudaEventDestroy(e.second);
        }
    for (void* p : c->allocs) cudaFree(p);
    delete c;
}

int dgfv_init_mesh(dgfv_ctx** out, const dgfv_mesh_desc* mesh, const dgfv_phys* phys, const dgfv_opts* opts) {
    if (!out || !mesh || !phys || !opts) return DGFV_ERR_ARG;
    *out = nullptr;
    if (mesh->n_domains < 1 || !mesh->dims || !mesh->lo || !mesh->hi) return DGFV_ERR_ARG;
    if (mesh->N_min < 1 || mesh->N_max > 7 || mesh->N_min > mesh->N_max) return DGFV_ERR_ARG;
    // N_fv = 0: per-element sub-cell counts (an FV element of degree N has N+1);
    // not with chained domains (mortars)
    const bool fv_own = mesh->N_fv == 0;
    if (fv_own && mesh->chain_x) return DGFV_ERR_ARG;
    const int nfv_max = fv_own ? mesh->N_max + 1 : mesh->N_fv;
    if (!fv_own && (mesh->N_fv < mesh->N_max + 1 || mesh->N_fv > MAXP)) return DGFV_ERR_ARG;
    // one FV element's sub-cell data must fit in the shared memory of one CTA
    if (fv_smem_bytes(phys->n_species, nfv_max) > 227 * 1024) return DGFV_ERR_ARG;
    if (phys->n_species < 1 || phys->n_species > 3) return DGFV_ERR_ARG;
    int64_t ne = 0;
    for (int d = 0; d < mesh->n_domains; ++d) {
        for (int a = 0; a < 3; ++a) {
            if (mesh->dims[3 * d + a] < 1 || !(mesh->hi[3 * d + a] > mesh->lo[3 * d + a])) return DGFV_ERR_ARG;
        }
        ne += (int64_t)mesh->dims[3 * d] * mesh->dims[3 * d + 1] * mesh->dims[3 * d + 2];
    }
    if (ne > (1LL << 30)) return DGFV_ERR_ARG;
    dgfv_ctx* c = new (std::nothrow) dgfv_ctx();
    if (!c) return DGFV_ERR_OOM;
    auto cleanup = [&](int r) {
        dgfv_destroy(c);
        return r;
    };
    if (cudaGetDevice(&c->dev) != cudaSuccess) return cleanup(DGFV_ERR_CUDA);
    if (cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->dev) != cudaSuccess)
        return cleanup(DGFV_ERR_CUDA);
    c->nk = phys->n_species;
    c->V = c->nk + 4;
    c->opts = *opts;
    c->N_min = mesh->N_min;
    c->N_max = mesh->N_max;
    c->nfv = nfv_max;  // the largest sub-cell count (capacities, shared memory)
    c->fv_own = fv_own;
    c->ph.nk = c->nk;
    if (opts->riemann < DGFV_RIEMANN_LLF || opts->riemann > DGFV_RIEMANN_HYBRID) return cleanup(DGFV_ERR_ARG);
    if (opts->nodes < 0 || opts->nodes > 1 || opts->split_form < 0 || opts->split_form > 1 ||
        (opts->split_form && opts->nodes != 1))
        return cleanup(DGFV_ERR_ARG);
    if (opts->integrator != DGFV_INTEGRATOR_SSPRK3 && opts->integrator != DGFV_INTEGRATOR_LSRK4)
        return cleanup(DGFV_ERR_ARG);
    c->ph.riemann = opts->riemann;
    c->ph.viscous = 0;
    c->ph.maxD = 0.0;
    for (int k = 0; k < c->nk; ++k) {
        if (!(phys->gamma[k] > 1.0) || !(phys->Rgas[k] > 0.0) || phys->mu[k] < 0 || phys->D[k] < 0 ||
            !(phys->Pr[k] > 0))
            return cleanup(DGFV_ERR_ARG);
        c->ph.cv[k] = phys->Rgas[k] / (phys->gamma[k] - 1.0);
        c->ph.cp[k] = phys->gamma[k] * c->ph.cv[k];
        c->ph.mu[k] = phys->mu[k];
        c->ph.pr[k] = phys->Pr[k];
        c->ph.D[k] = phys->D[k];
        c->ph.maxD = std::max(c->ph.maxD, phys->D[k]);
        if (phys->mu[k] != 0.0 || phys->D[k] != 0.0) c->ph.viscous = 1;
    }
    c->ph.sutherland = phys->sutherland ? 1 : 0;
    c->ph.T_ref = phys->T_ref;
    c->ph.S = phys->S;
    if (c->ph.sutherland && !(phys->T_ref > 0.0 && phys->S >= 0.0)) return cleanup(DGFV_ERR_ARG);
    if (opts->indicator_vars < 0 || opts->indicator_vars > 1) return cleanup(DGFV_ERR_ARG);
    if (opts->pp_limiter < 0 || opts->pp_limiter > 1 || (opts->pp_limiter && !(opts->pp_eps > 0.0)))
        return cleanup(DGFV_ERR_ARG);
    c->n_elem = (int)ne;
    c->nb.resize(6 * ne);
    c->rh.resize(3 * ne);
    std::vector<int64_t> first(mesh->n_domains + 1, 0);
    for (int dm = 0; dm < mesh->n_domains; ++dm) {
        const int dims[3] = {mesh->dims[3 * dm], mesh->dims[3 * dm + 1], mesh->dims[3 * dm + 2]};
        const int64_t e0 = first[dm];
        double rh[3];
        for (int a = 0; a < 3; ++a) rh[a] = 2.0 * dims[a] / (mesh->hi[3 * dm + a] - mesh->lo[3 * dm + a]);
        for (int k = 0; k < dims[2]; ++k)
            for (int j = 0; j < dims[1]; ++j)
                for (int i = 0; i < dims[0]; ++i) {
                    const int64_t e = e0 + i + (int64_t)dims[0] * (j + (int64_t)dims[1] * k);
                    const int ijk[3] = {i, j, k};
                    for (int f = 0; f < 6; ++f) {
                        int q[3] = {i, j, k};
                        const int a = f / 2;
                        q[a] = (ijk[a] + ((f & 1) ? 1 : -1) + dims[a]) % dims[a];
                        c->nb[6 * e + f] = (int32_t)(e0 + q[0] + (int64_t)dims[0] * (q[1] + (int64_t)dims[1] * q[2]));
                    }
                    for (int a = 0; a < 3; ++a) c->rh[3 * e + a] = rh[a];
                }
        first[dm + 1] = e0 + (int64_t)dims[0] * dims[1] * dims[2];
    }
    if (mesh->chain_x != 0 && mesh->chain_x != 1) return cleanup(DGFV_ERR_ARG);
    if (mesh->chain_x) {
        // Sec. 3.2.3: domain A's +x side against domain A+1's -x side (cyclic);
        // equal (ny, nz): conforming; 2:1 in one or both: mortars, big sides on
        // the coarser domain.  Each mortar face of an element gets a slot.
        const int D = mesh->n_domains;
        for (int A = 0; A < D; ++A)
            for (int a = 1; a < 3; ++a)
                if (mesh->lo[3 * A + a] != mesh->lo[a] || mesh->hi[3 * A + a] != mesh->hi[a]) return cleanup(DGFV_ERR_ARG);
        auto elem = [&](int dm, int i, int j, int k) {
            const int32_t* dd = mesh->dims + 3 * dm;
            return (int32_t)(first[dm] + i + (int64_t)dd[0] * (j + (int64_t)dd[1] * k));
        };
        auto ratio = [](int x, int y) { return x == y ? 0 : (y == 2 * x ? 1 : (x == 2 * y ? -1 : 9)); };
        for (int A = 0; A < D; ++A) {
            const int Bd = (A + 1) % D;
            const int32_t *da = mesh->dims + 3 * A, *db = mesh->dims + 3 * Bd;
            const int ra = ratio(da[1], db[1]), rb = ratio(da[2], db[2]);
            if (ra == 9 || rb == 9 || ra * rb < 0) return cleanup(DGFV_ERR_ARG);
            if (ra == 0 && rb == 0) {
                for (int k = 0; k < da[2]; ++k)
                    for (int j = 0; j < da[1]; ++j) {
                        const int32_t eA = elem(A, da[0] - 1, j, k), eB = elem(Bd, 0, j, k);
                        c->nb[6 * (int64_t)eA + 1] = eB;
                        c->nb[6 * (int64_t)eB + 0] = eA;
                    }
                continue;
            }
            const bool bigA = ra > 0 || rb > 0;
            const int Dg = bigA ? A : Bd, Ds = bigA ? Bd : A;
            const int32_t *dg = mesh->dims + 3 * Dg, *ds = mesh->dims + 3 * Ds;
            const int fB = bigA ? 1 : 0, sa = ra != 0, sb = rb != 0;
            for (int k = 0; k < dg[2]; ++k)
                for (int j = 0; j < dg[1]; ++j) {
                    const int m = c->n_mort++;
                    const int32_t eb = elem(Dg, bigA ? dg[0] - 1 : 0, j, k);
                    c->m_big.push_back(eb);
                    c->m_fB.push_back((uint8_t)fB);
                    c->m_split.push_back((uint8_t)(sa | (sb << 1)));
                    c->m_vfirst.push_back(c->n_virt);
                    int32_t first_small = -1;
                    for (int qb = 0; qb <= sb; ++qb)
                        for (int qa = 0; qa <= sa; ++qa) {
                            const int32_t es = elem(Ds, bigA ? 0 : ds[0] - 1, sa ? 2 * j + qa : j, sb ? 2 * k + qb : k);
                            if (first_small < 0) first_small = es;
                            c->v_mort.push_back(m);
                            c->v_quad.push_back((uint8_t)(qa + 2 * qb));
                            c->v_small.push_back(es);
                            c->n_virt++;
                            c->nb[6 * (int64_t)es + (fB ^ 1)] = -1 - c->n_slot++;
                            c->s_elem.push_back(es);
                            c->s_face.push_back((uint8_t)(fB ^ 1));
                            c->s_mort.push_back(m);
                            c->s_quad.push_back((int8_t)(qa + 2 * qb));
                            c->s_nbe.push_back(eb);
                        }
                    c->nb[6 * (int64_t)eb + fB] = -1 - c->n_slot++;
                    c->s_elem.push_back(eb);
                    c->s_face.push_back((uint8_t)fB);
                    c->s_mort.push_back(m);
                    c->s_quad.push_back(-1);
                    c->s_nbe.push_back(first_small);
                }
        }
        c->m_vfirst.push_back(c->n_virt);
    }
    // faces: every +a face of an element with an element across (conforming),
    // then every virtual small side against its small element (x faces)
    for (int64_t e = 0; e < ne; ++e)
        for (int a = 0; a < 3; ++a) {
            const int32_t q = c->nb[6 * e + 2 * a + 1];
            if (q < 0) continue;
            c->faceL.push_back((int32_t)e);
            c->faceR.push_back(q);
            c->faceD.push_back((uint8_t)a);
        }
    for (int v = 0; v < c->n_virt; ++v) {
        const int32_t ev = (int32_t)(ne + v), es = c->v_small[v];
        const bool big_lower = c->m_fB[c->v_mort[v]] == 1;
        c->faceL.push_back(big_lower ? ev : es);
        c->faceR.push_back(big_lower ? es : ev);
        c->faceD.push_back(0);
    }
    c->n_faces = (int)c->faceL.size();
    // capacity: every element at the largest point count
    const int nmax = std::max(c->N_max + 1, c->nfv);
    c->cap_state = ne * (int64_t)c->V * nmax * nmax * nmax;
    c->cap_fpts = (ne + c->n_virt) * 6LL * nmax * nmax;
    const int64_t nt = ne + c->n_virt;
    int r = DGFV_OK;
#define A_(p, n)                                 \
    if ((r = dalloc(c, &(p), (size_t)(n))) != DGFV_OK) return cleanup(r);
    A_(c->d_n, nt) A_(c->d_N, nt) A_(c->d_fv, nt) A_(c->d_off, ne) A_(c->d_fo, nt)
    A_(c->d_m_big, c->n_mort) A_(c->d_m_fB, c->n_mort) A_(c->d_m_split, c->n_mort) A_(c->d_m_vfirst, c->n_mort + 1)
    A_(c->d_v_mort, c->n_virt) A_(c->d_v_quad, c->n_virt) A_(c->d_v_small, c->n_virt)
    A_(c->d_s_elem, c->n_slot) A_(c->d_s_face, c->n_slot) A_(c->d_s_mort, c->n_slot) A_(c->d_s_quad, c->n_slot)
    A_(c->d_s_nbe, c->n_slot) A_(c->d_s_active, c->n_slot) A_(c->d_mnb, (int64_t)c->n_slot * c->V * c->nfv * c->nfv)
    A_(c->d_n_old, ne) A_(c->d_N_old, ne) A_(c->d_fv_old, ne) A_(c->d_off_old, ne)
    A_(c->d_nb, 6 * ne) A_(c->d_rh, 3 * ne)
    A_(c->d_faceL, c->n_faces) A_(c->d_faceR, c->n_faces) A_(c->d_faceD, c->n_faces)
    A_(c->d_fu, c->cap_fpts * c->V) A_(c->d_fg, c->cap_fpts * 3 * c->V) A_(c->d_flux, c->cap_fpts * c->V)
    A_(c->d_flift, c->cap_fpts * c->V) A_(c->d_frec, c->cap_fpts * c->V)
    A_(c->d_rtmp, c->cap_state) A_(c->d_U, c->cap_state) A_(c->d_Us, c->cap_state)
    A_(c->d_dt3, 4) A_(c->d_partial, 2 * ne + 2) A_(c->d_Ip, ne) A_(c->d_Ih, ne) A_(c->d_dec, ne)
    A_(c->d_status, 2) A_(c->d_queue, 1) A_(c->d_pp_count, 2) A_(c->lift.d, c->n_faces) A_(c->flux.d, c->n_faces)
    A_(c->conf.d_first, c->n_faces) A_(c->conf.d_count, c->n_faces) A_(c->conf.d_nc, c->n_faces)
    A_(c->conf.d_d, c->n_faces) A_(c->conf.d_items, c->n_faces)
    A_(c->mixed.tiles.d_first, c->n_faces) A_(c->mixed.tiles.d_count, c->n_faces)
    A_(c->mixed.tiles.d_nc, c->n_faces) A_(c->mixed.tiles.d_d, c->n_faces) A_(c->mixed.tiles.d_items, c->n_faces)
    A_(c->mixed.d_face, c->n_faces) A_(c->mixed.d_pt, c->n_faces)
#undef A_
    if ((r = alloc_tiles(c, c->all)) != DGFV_OK) return cleanup(r);
    if ((r = alloc_tiles(c, c->dg)) != DGFV_OK) return cleanup(r);
    if ((r = alloc_tiles(c, c->fvt)) != DGFV_OK) return cleanup(r);
    if (cudaMemset(c->d_status, 0, 2 * sizeof(int)) != cudaSuccess) return cleanup(DGFV_ERR_CUDA);
    if (cudaMemset(c->d_pp_count, 0, 2 * sizeof(unsigned long long)) != cudaSuccess) return cleanup(DGFV_ERR_CUDA);
    if (cudaMemcpy(c->d_nb, c->nb.data(), c->nb.size() * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->d_rh, c->rh.data(), c->rh.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->d_faceL, c->faceL.data(), c->n_faces * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->d_faceR, c->faceR.data(), c->n_faces * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->d_faceD, c->faceD.data(), c->n_faces, cudaMemcpyHostToDevice) != cudaSuccess)
        return cleanup(DGFV_ERR_CUDA);
    if (c->n_mort) {
        auto up = [](void* d, const void* h, size_t bytes) { return cudaMemcpy(d, h, bytes, cudaMemcpyHostToDevice); };
        if (up(c->d_m_big, c->m_big.data(), c->n_mort * 4) != cudaSuccess ||
            up(c->d_m_fB, c->m_fB.data(), c->n_mort) != cudaSuccess ||
            up(c->d_m_split, c->m_split.data(), c->n_mort) != cudaSuccess ||
            up(c->d_m_vfirst, c->m_vfirst.data(), (c->n_mort + 1) * 4) != cudaSuccess ||
            up(c->d_v_mort, c->v_mort.data(), c->n_virt * 4) != cudaSuccess ||
            up(c->d_v_quad, c->v_quad.data(), c->n_virt) != cudaSuccess ||
            up(c->d_v_small, c->v_small.data(), c->n_virt * 4) != cudaSuccess ||
            up(c->d_s_elem, c->s_elem.data(), c->n_slot * 4) != cudaSuccess ||
            up(c->d_s_face, c->s_face.data(), c->n_slot) != cudaSuccess ||
            up(c->d_s_mort, c->s_mort.data(), c->n_slot * 4) != cudaSuccess ||
            up(c->d_s_quad, c->s_quad.data(), c->n_slot) != cudaSuccess ||
            up(c->d_s_nbe, c->s_nbe.data(), c->n_slot * 4) != cudaSuccess)
            return cleanup(DGFV_ERR_CUDA);
    }
    try {
        if ((r = build_bank(c)) != DGFV_OK) return cleanup(r);
    } catch (...) {
        return cleanup(DGFV_ERR_ARG);
    }
    c->N.assign(nt, (uint8_t)c->N_min);
    c->fv.assign(nt, 0);
    if ((r = apply_layout(c)) != DGFV_OK) return cleanup(r);
    *out = c;
    return DGFV_OK;
}

int64_t dgfv_num_elements(const dgfv_ctx* c) { return c ? c->n_elem : -1; }

int dgfv_set_degrees(dgfv_ctx* c, const int8_t* N, const uint8_t* is_fv, int remap_state) {
    const NvtxRange nvtx_range("dgfv_set_degrees");
    if (!c || !N) return DGFV_ERR_ARG;
    TRY(check_dev(c));
    return set_pattern(c, N, is_fv, remap_state != 0, nullptr);
}

int dgfv_get_degrees(dgfv_ctx* c, int8_t* N, uint8_t* is_fv) {
    if (!c) return DGFV_ERR_ARG;
    for (int e = 0; e < c->n_elem; ++e) {
        if (N) N[e] = (int8_t)c->N[e];
        if (is_fv) is_fv[e] = c->fv[e];
    }
    return DGFV_OK;
}

int dgfv_state_layout(dgfv_ctx* c, int64_t* n_doubles, const int64_t** d_elem_offsets) {
    if (!c) return DGFV_ERR_ARG;
    if (n_doubles) *n_doubles = c->n_state;
    if (d_elem_offsets) *d_elem_offsets = c->d_off;
    return DGFV_OK;
}

// The device address of page-locked host memory (cudaHostAlloc,
// cudaHostRegister), or null for pageable memory.
static void* host_device_view(const void* h) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, h) != cudaSuccess) {
        cudaGetLastError();  // clear: an unknown pointer is pageable memory here
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// State copies.  Host buffers in page-locked memory are copied by a kernel on
// every SM through their device mapping, pageable ones by cudaMemcpyAsync.
// Measured on a GB300 (Grace host, 64 KB pages, 715 MB of state): after a
// cycle of GPU work the copy engines took 24-43 ms for the first copy of the
// buffer and 3.6-4.0 ms when it was repeated at once (the device's
// translations of the buffer's host pages are refilled in sequence), the SM
// copy 3.8-4.5 ms in both cases.
static int copy_state(dgfv_ctx* c, void* dst, const void* src, int64_t n, cudaMemcpyKind kind, void* stream,
                      bool sync) {
    if (!c || (!dst && n > 0) || (!src && n > 0)) return DGFV_ERR_ARG;
    TRY(check_dev(c));
    if (n != c->n_state) return fail(c, DGFV_ERR_ARG, "state size does not match the layout");
    cudaStream_t s = (cudaStream_t)stream;
    void* hv = nullptr;
    if (n > 0 && kind == cudaMemcpyHostToDevice) hv = host_device_view(src);
    if (n > 0 && kind == cudaMemcpyDeviceToHost) hv = host_device_view(dst);
    if (hv) {
        if (kind == cudaMemcpyHostToDevice)
            launch_copy_state(static_cast<double*>(dst), static_cast<const double*>(hv), n, c->n_sm, s);
        else
            launch_copy_state(static_cast<double*>(hv), static_cast<const double*>(src), n, c->n_sm, s);
        CK(cudaGetLastError());
    } else {
        CK(cudaMemcpyAsync(dst, src, n * sizeof(double), kind, s));
    }
    if (sync) CK(cudaStreamSynchronize(s));
    return DGFV_OK;
}

int dgfv_set_state(dgfv_ctx* c, const double* d_U, int64_t n, void* stream) {
    int r = copy_state(c, c ? c->d_U : nullptr, d_U, n, cudaMemcpyDeviceToDevice, stream, false);
    if (r == DGFV_OK) c->state_valid = true;
    return r;
}

int dgfv_get_state(dgfv_ctx* c, double* d_U, int64_t n, void* stream) {
    if (c && !c->state_valid) return fail(c, DGFV_ERR_STATE, "no state set");
    return copy_state(c, d_U, c ? c->d_U : nullptr, n, cudaMemcpyDeviceToDevice, stream, false);
}

int dgfv_set_state_host(dgfv_ctx* c, const double* h_U, int64_t n, void* stream) {
    int r = copy_state(c, c ? c->d_U : nullptr, h_U, n, cudaMemcpyHostToDevice, stream, true);
    if (r == DGFV_OK) c->state_valid = true;
    return r;
}

int dgfv_get_state_host(dgfv_ctx* c, double* h_U, int64_t n, void* stream) {
    if (c && !c->state_valid) return fail(c, DGFV_ERR_STATE, "no state set");
    return copy_state(c, h_U, c ? c->d_U : nullptr, n, cudaMemcpyDeviceToHost, stream, true);
}

int dgfv_eval_rhs(dgfv_ctx* c, const double* d_U, double* d_R, void* stream) {
    const NvtxRange nvtx_range("dgfv_eval_rhs");
    if (!c || !d_U || !d_R) return DGFV_ERR_ARG;
    TRY(check_dev(c));
    if (d_U == d_R) return fail(c, DGFV_ERR_ARG, "d_U and d_R alias");
    cudaStream_t s = (cudaStream_t)stream;
    enqueue_stage(c, d_U, d_U, d_R, 0, 0.0, 0.0, s);
    CK(cudaGetLastError());
    return DGFV_OK;
}

int dgfv_compute_dt(dgfv_ctx* c, const double* d_U, double* out3, void* stream) {
    const NvtxRange nvtx_range("dgfv_compute_dt");
    if (!c || !d_U || !out3) return DGFV_ERR_ARG;
    TRY(check_dev(c));
    cudaStream_t s = (cudaStream_t)stream;
    launch_dt(c->nk, params(c), c->all.view(), c->all.ntiles, d_U, c->opts.cfl_c, c->opts.cfl_v, c->d_partial,
              c->d_dt3, s);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out3, c->d_dt3, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return DGFV_OK;
}

int dgfv_compute_dt_noalloc(dgfv_ctx* c, const double* d_U, double* d_out3, void* stream) {
    if (!c || !d_U || !d_out3) return DGFV_ERR_ARG;
    TRY(check_dev(c));
    const int r = launch_dt_noalloc(c->nk, params(c), c->all.view(), c->all.ntiles, d_U, c->opts.cfl_c,
                                    c->opts.cfl_v, d_out3, (cudaStream_t)stream);
    if (r == 1)
        return fail(c, DGFV_ERR_ARG, "dgfv_compute_dt_noalloc: " + std::to_string(c->all.ntiles) +
                                         " work tiles exceed the fixed scratch of " +
                                         std::to_string(DT_NOALLOC_MAX_BLOCKS) + " blocks");
    if (r != 0) return fail(c, DGFV_ERR_CUDA, "dgfv_compute_dt_noalloc: CUDA error");
    return DGFV_OK;
}

static int adj_prepare(dgfv_ctx* c) {
    if (c->adj_ready) return DGFV_OK;
    TRY(dalloc(c, &c->d_fbar, c->cap_fpts * c->V));
    TRY(dalloc(c, &c->d_ubar, c->cap_fpts * c->V));
    TRY(dalloc(c, &c->d_gbar, c->cap_fpts * 3 * c->V));
    TRY(dalloc(c, &c->d_sbar, c->cap_fpts * c->V));
    TRY(dalloc(c, &c->d_S1, c->cap_state));
    TRY(dalloc(c, &c->d_S2, c->cap_state));
    TRY(dalloc(c, &c->d_B1, c->cap_state));
    TRY(dalloc(c, &c->d_B2, c->cap_state));
    TRY(dalloc(c, &c->d_W, c->cap_state));
    TRY(dalloc(c, &c->d_gvol, 3 * c->cap_state));
    TRY(dalloc(c, &c->d_gf, 6 * c->cap_state));
    TRY(dalloc(c, &c->d_fvs, 2 * c->cap_state));
    c->adj_ready = true;
    return DGFV_OK;
}

// U_bar = (dR/dU)^T R_bar at U (Ub must not alias U or Rb).
static void enqueue_vjp(dgfv_ctx* c, const double* U, const double* Rb, double* Ub, cudaStream_t s) {
    const Params P = params(c);
    const Faces F{c->d_faceL, c->d_faceR, c->d_faceD};
    const AdjBuffers A{c->d_fbar, c->d_ubar, c->d_gbar, c->d_sbar};
    const MortarTables MT = mortar_tables(c);
    // forward face values and lifting values of U (mortars: the virtual small
    // sides' values, the big sides' projected lifting values)
    launch_prolong(c->nk, P, c->all.view(), c->all.ntiles, U, s);
    if (c->n_fv_elems) {  // FV face states and gradients (with the neighbour values across mortars)
        launch_mortar_nb(c->nk, P, MT, c->d_s_active, c->n_slot_active, U, c->d_mnb, s);
        launch_fv(c->nk, P, c->fvt.view(), c->fvt.ntiles, U, s, true, c->fv_variant);
    }
    launch_mortar_in(c->nk, P, MT, c->n_virt, 0, s);
    if (c->ph.viscous) {
        launch_face_lift(c->nk, P, F, c->lift.d, c->lift.count, s);
        launch_mortar_out(c->nk, P, MT, c->n_mort, 0, s);
    }
    launch_adj_surface(c->nk, P, A, c->dg.view(), c->dg.ntiles, Rb, s);
    launch_adj_surface_fv(c->nk, P, A, c->fvt.view(), c->fvt.ntiles, Rb, s);
    launch_adj_mortar_virt(c->nk, P, A, MT, c->n_virt, 0, s);
    // recomputed gradient (and its traces), volume integral^T, nodal reverse
    launch_adj_vol_a(c->nk, P, c->dg.view(), c->dg.ntiles, c->adj_smem, U, Rb, Ub, c->d_gvol, c->d_gf, s,
                     c->opts.split_form);
    if (c->opts.split_form) launch_adj_split(c->nk, P, c->dg.view(), c->dg.ntiles, c->adj_split_smem, U, Rb, Ub, s);
    if (c->ph.viscous) launch_mortar_in(c->nk, P, MT, c->n_virt, 1, s);
    launch_adj_faces(c->nk, P, A, F, c->conf.view(), c->conf.ntiles, s);
    launch_adj_mixed_faces(c->nk, P, A, F, c->mixed.tiles.view(), c->mixed.tiles.ntiles, c->mixed.d_face,
                           c->mixed.d_pt, c->mixed.n, c->mixed.d_in, c->mixed.d_out, s);
    if (c->ph.viscous) {
        launch_adj_mortar_big(c->nk, P, A, MT, c->n_mort, 0, s);
        launch_adj_vol_b(c->nk, P, A, c->dg.view(), c->dg.ntiles, c->dg.smem, c->d_gvol, Ub, s);
        launch_adj_mortar_virt(c->nk, P, A, MT, c->n_virt, 1, s);
        launch_adj_lift(c->nk, P, A, F, c->lift.d, c->lift.count, s);
    }
    launch_adj_mortar_big(c->nk, P, A, MT, c->n_mort, 1, s);
    if (c->n_fv_elems) {
        launch_adj_fv_elements(c->nk, P, A, c->fvt.view(), c->fvt.ntiles, U, Rb, Ub, c->d_gf, c->d_gvol, c->d_fvs,
                               c->cap_state, c->n_elem, s);
        launch_adj_mortar_nb(c->nk, P, A, MT, c->n_mort, Ub, s);
    }
    launch_adj_prolong(c->nk, P, A, c->dg.view(), c->dg.ntiles, Ub, s);
}

int dgfv_rhs_vjp(dgfv_ctx* c, const double* d_U, const double* d_Rbar, double* d_Ubar, void* stream) {
    const NvtxRange nvtx_range("dgfv_rhs_vjp");
    if (!c || !d_U || !d_Rbar || !d_Ubar) return DGFV_ERR_ARG;
    TRY(check_dev(c));
    if (d_Ubar == d_U || d_Ubar == d_Rbar) return fail(c, DGFV_ERR_ARG, "d_Ubar aliases an input");
    TRY(adj_prepare(c));
    enqueue_vjp(c, d_U, d_Rbar, d_Ubar, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return DGFV_OK;
}

static int rk_step_vjp_impl(dgfv_ctx* c, const double* d_U0, const double* d_U1, const double* d_U2, double dt,
                            const double* d_Ubar_next, double* d_Ubar, cudaStream_t s) {
    const int64_t n = c->n_state;
    // U3 = 1/3 U0 + 2/3 (U2 + dt R(U2)), backwards (W = J^T of the stage's adjoint):
    enqueue_vjp(c, d_U2, d_Ubar_next, c->d_W, s);
    // U2_bar = 2/3 (U3_bar + dt W);  U0_bar = 1/3 U3_bar
    launch_rk3_adj_combine(n, 0, 2.0 / 3.0, 1.0 / 3.0, dt, d_Ubar_next, c->d_W, c->d_B2, d_Ubar, s);
    enqueue_vjp(c, d_U1, c->d_B2, c->d_W, s);
    // U1_bar = 1/4 (U2_bar + dt W);  U0_bar += 3/4 U2_bar
    launch_rk3_adj_combine(n, 1, 0.25, 0.75, dt, c->d_B2, c->d_W, c->d_B1, d_Ubar, s);
    enqueue_vjp(c, d_U0, c->d_B1, c->d_W, s);
    // U0_bar += U1_bar + dt W
    launch_rk3_adj_combine(n, 2, 0.0, 0.0, dt, c->d_B1, c->d_W, nullptr, d_Ubar, s);
    CK(cudaGetLastError());
    return DGFV_OK;
}

// Adjoint of one low-storage RK4 step from U0, the stage states recomputed:
// forward U_s = U_{s-1} + B_s dU_s, dU_s = A_s dU_{s-1} + dt R(U_{s-1});
// backwards, with dU_bar = 0 after the step:
//   dU_bar_s += B_s U_bar_s;  U_bar_{s-1} = U_bar_s + dt J(U_{s-1})^T dU_bar_s;
//   dU_bar_{s-1} = A_s dU_bar_s.
// U_1..U_4 live in the four adjoint stage buffers, dU_bar in the context's
// low-storage register (free between steps).
static int lsrk4_step_vjp(dgfv_ctx* c, const double* d_U0, double dt, const double* d_Ubar_next, double* d_Ubar,
                          cudaStream_t s) {
    const int64_t n = c->n_state;
    const double* Us[5] = {d_U0, c->d_S1, c->d_S2, c->d_B1, c->d_B2};
    launch_set_scalar(c->d_dt3, dt, s);
    for (int st = 0; st < 4; ++st)
        enqueue_stage(c, Us[st], Us[st], const_cast<double*>(Us[st + 1]), 2, LSRK4_A[st], LSRK4_B[st], s, st > 0,
                      st < 3);
    double* dUb = c->d_Us;
    launch_axpby(n, 1.0, d_Ubar_next, 0.0, d_Ubar_next, d_Ubar, s);                  // U_bar_5
    for (int st = 4; st >= 0; --st) {
        if (st == 4)
            launch_axpby(n, LSRK4_B[4], d_Ubar, 0.0, d_Ubar, dUb, s);                // dU_bar_5 = B_5 U_bar_5
        else
            launch_axpby(n, 1.0, dUb, LSRK4_B[st], d_Ubar, dUb, s);
        enqueue_vjp(c, Us[st], dUb, c->d_W, s);
        launch_axpby(n, 1.0, d_Ubar, dt, c->d_W, d_Ubar, s);
        if (st > 0) launch_axpby(n, LSRK4_A[st], dUb, 0.0, dUb, dUb, s);
    }
    CK(cudaGetLastError());
    return DGFV_OK;
}

int dgfv_rk_step_vjp(dgfv_ctx* c, const double* d_U0, double dt, const double* d_Ubar_next, double* d_Ubar,
                     void* stream) {
    const NvtxRange nvtx_range("dgfv_rk_step_vjp");
    if (!c || !d_U0 || !d_Ubar_next || !d_Ubar || !(dt > 0.0)) return DGFV_ERR_ARG;
    TRY(check_dev(c));
    if (d_Ubar == d_Ubar_next || d_Ubar == d_U0) return fail(c, DGFV_ERR_ARG, "d_Ubar aliases an input");
    if (c->opts.pp_limiter) return fail(c, DGFV_ERR_ARG, "step adjoints do not support the positivity limiter");
    TRY(adj_prepare(c));
    cudaStream_t s = (cudaStream_t)stream;
    if (c->opts.integrator == DGFV_INTEGRATOR_LSRK4) return lsrk4_step_vjp(c, d_U0, dt, d_Ubar_next, d_Ubar, s);
    // stage states of the step (recomputed from the step's start state)
    launch_set_scalar(c->d_dt3, dt, s);
    enqueue_stage(c, d_U0, d_U0, c->d_S1, 1, 0.0, 1.0, s, false, true);      // U1 = U0 + dt R(U0)
    enqueue_stage(c, c->d_S1, d_U0, c->d_S2, 1, 0.75, 0.25, s, true, false);  // U2 = 3/4 U0 + 1/4 (U1 + dt R(U1))
    return rk_step_vjp_impl(c, d_U0, c->d_S1, c->d_S2, dt, d_Ubar_next, d_Ubar, s);
}

int dgfv_rk_step_vjp_stages(dgfv_ctx* c, const double* const* d_stages, double dt, const double* d_Ubar_next,
                            double* d_Ubar, void* stream) {
    const NvtxRange nvtx_range("dgfv_rk_step_vjp_stages");
    if (!c || !d_stages || !d_stages[0] || !d_stages[1] || !d_stages[2] || !d_Ubar_next || !d_Ubar || !(dt > 0.0))
        return DGFV_ERR_ARG;
    TRY(check_dev(c));
    for (int i = 0; i < 3; ++i)
        if (d_Ubar == d_stages[i]) return fail(c, DGFV_ERR_ARG, "d_Ubar aliases an input");
    if (d_Ubar == d_Ubar_next) return fail(c, DGFV_ERR_ARG, "d_Ubar aliases an input");
    if (c->opts.integrator != DGFV_INTEGRATOR_SSPRK3 || c->opts.pp_limiter)
        return fail(c, DGFV_ERR_ARG, "stage adjoints and stage saving support SSP-RK3 without the limiter only");
    TRY(adj_prepare(c));
    return rk_step_vjp_impl(c, d_stages[0], d_stages[1], d_stages[2], dt, d_Ubar_next, d_Ubar, (cudaStream_t)stream);
}

int dgfv_rk_step_save(dgfv_ctx* c, double dt, double* d_stage1, double* d_stage2, void* stream) {
    const NvtxRange nvtx_range("dgfv_rk_step_save");
    if (!c || !d_stage1 || !d_stage2 || !(dt > 0.0)) return DGFV_ERR_ARG;
    TRY(check_dev(c));
    if (!c->state_valid) return fail(c, DGFV_ERR_STATE, "rk_step_save before set_state");
    if (c->opts.integrator != DGFV_INTEGRATOR_SSPRK3 || c->opts.pp_limiter)
        return fail(c, DGFV_ERR_ARG, "stage adjoints and stage saving support SSP-RK3 without the limiter only");
    cudaStream_t s = (cudaStream_t)stream;
    launch_set_scalar(c->d_dt3, dt, s);
    enqueue_stage(c, c->d_U, c->d_U, d_stage1, 1, 0.0, 1.0, s, false, true);
    enqueue_stage(c, d_stage1, c->d_U, d_stage2, 1, 0.75, 0.25, s, true, true);
    enqueue_stage(c, d_stage2, c->d_U, c->d_U, 1, 1.0 / 3.0, 2.0 / 3.0, s, true, false);
    CK(cudaGetLastError());
    return DGFV_OK;
}

int dgfv_rk_step(dgfv_ctx* c, double dt, double* dt_used, void* stream) {
    const NvtxRange nvtx_range("dgfv_rk_step");
    if (!c) return DGFV_ERR_ARG;
    TRY(check_dev(c));
    if (!c->state_valid) return fail(c, DGFV_ERR_STATE, "rk_step before set_state");
    cudaStream_t s = (cudaStream_t)stream;
    enqueue_rk_step(c, dt, s);
    CK(cudaGetLastError());
    if (dt_used) {
        CK(cudaMemcpyAsync(dt_used, c->d_dt3, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        return read_status(c, s);
    }
    return DGFV_OK;
}

int dgfv_rk_steps(dgfv_ctx* c, int n_steps, double dt, double* dt_used, void* stream) {
    const NvtxRange nvtx_range("dgfv_rk_steps");
    if (!c || n_steps < 0) return DGFV_ERR_ARG;
    TRY(check_dev(c));
    if (!c->state_valid) return fail(c, DGFV_ERR_STATE, "rk_steps before set_state");
    cudaStream_t s = (cudaStream_t)stream;
    if (c->prof.on) {
        for (int i = 0; i < n_steps; ++i) enqueue_rk_step(c, dt, s);
        CK(cudaGetLastError());
    } else if (!c->graph_valid || c->graph_dt != dt || c->graph_stream != s) {
        if (c->graph) {
            cudaGraphExecDestroy(c->graph);
            c->graph = nullptr;
        }
        cudaStream_t cs;
        CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g;
        CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        enqueue_rk_step(c, dt, cs);
        cudaError_t e = cudaStreamEndCapture(cs, &g);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) return fail(c, DGFV_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&c->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(c, DGFV_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        c->graph_valid = true;
        c->graph_dt = dt;
        c->graph_stream = s;
    }
    if (!c->prof.on)
        for (int i = 0; i < n_steps; ++i) CK(cudaGraphLaunch(c->graph, s));
    if (dt_used) {
        CK(cudaMemcpyAsync(dt_used, c->d_dt3, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        return read_status(c, s);
    }
    return DGFV_OK;
}

int dgfv_indicator(dgfv_ctx* c, const double* d_U, double* d_Ip, double* d_Ih, uint8_t* d_decision, void* stream) {
    if (!c || !d_U) return DGFV_ERR_ARG;
    TRY(check_dev(c));
    const double thr[4] = {c->opts.T_fv_on, c->opts.T_fv_off, c->opts.T_ref, c->opts.T_crs};
    Timed t(c, K_INDICATOR, (cudaStream_t)stream);
    launch_indicator(c->nk, params(c), d_U, c->n_elem, d_Ip, d_Ih, d_decision, thr, c->N_min, c->N_max,
                     c->opts.indicator_vars,
                     (cudaStream_t)stream);
    CK(cudaGetLastError());
    return DGFV_OK;
}

int dgfv_adapt(dgfv_ctx* c, dgfv_adapt_stats* stats, void* stream) {
    const NvtxRange nvtx_range("dgfv_adapt");
    if (!c) return DGFV_ERR_ARG;
    TRY(check_dev(c));
    if (!c->state_valid) return fail(c, DGFV_ERR_STATE, "adapt before set_state");
    cudaStream_t s = (cudaStream_t)stream;
    TRY(dgfv_indicator(c, c->d_U, c->d_Ip, c->d_Ih, c->d_dec, stream));
    std::vector<uint8_t> dec(c->n_elem);
    std::vector<double> Ip(c->n_elem), Ih(c->n_elem);
    CK(cudaMemcpyAsync(dec.data(), c->d_dec, c->n_elem, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(Ip.data(), c->d_Ip, c->n_elem * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(Ih.data(), c->d_Ih, c->n_elem * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<int8_t> Nn(c->n_elem);
    std::vector<uint8_t> fn(c->n_elem);
    int64_t changed = 0, near = 0;
    const double T[4] = {c->opts.T_fv_on, c->opts.T_fv_off, c->opts.T_ref, c->opts.T_crs};
    for (int e = 0; e < c->n_elem; ++e) {
        int N = c->N[e];
        int f = c->fv[e];
        switch (dec[e]) {
            case 1: f = 1; break;
            case 2: f = 0; break;
            case 3: N = N + 1; break;
            case 4: N = N - 1; break;
            default: break;
        }
        Nn[e] = (int8_t)N;
        fn[e] = (uint8_t)f;
        changed += dec[e] != 0;
        bool nr = std::fabs(Ih[e] - (c->fv[e] ? T[1] : T[0])) < 1e-10;
        if (!c->fv[e]) nr = nr || std::fabs(Ip[e] - T[2]) < 1e-10 || std::fabs(Ip[e] - T[3]) < 1e-10;
        near += nr;
    }
    if (changed) TRY(set_pattern(c, Nn.data(), fn.data(), true, s));
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        int64_t dofs = 0;
        for (int e = 0; e < c->n_elem; ++e) {
            if (c->fv[e]) stats->n_fv++;
            else stats->hist[c->N[e]]++;
            dofs += (int64_t)c->npts[e] * c->npts[e] * c->npts[e];
        }
        stats->n_changed = changed;
        stats->n_near = near;
        stats->mean_dofs = (double)dofs / c->n_elem;
    }
    return read_status(c, s);
}

int dgfv_profile_enable(dgfv_ctx* c, int on) {
    if (!c) return DGFV_ERR_ARG;
    CK(cudaDeviceSynchronize());
    c->prof.on = on != 0;
    for (int k = 0; k < K_COUNT; ++k) c->prof.used[k] = 0;
    return DGFV_OK;
}

int dgfv_profile_read(dgfv_ctx* c, double* ms, int64_t* launches, int cap) {
    if (!c || cap < 0) return DGFV_ERR_ARG;
    CK(cudaDeviceSynchronize());
    const int nk = std::min<int>(cap, K_COUNT);
    for (int k = 0; k < nk; ++k) {
        double tot = 0.0;
        for (size_t i = 0; i < c->prof.used[k]; ++i) {
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, c->prof.ev[k][i].first, c->prof.ev[k][i].second));
            tot += t;
        }
        if (ms) ms[k] = tot;
        if (launches) launches[k] = (int64_t)c->prof.used[k];
    }
    return nk;
}

int dgfv_set_launch_mode(dgfv_ctx* c, int mode) {
    if (!c || mode < 0 || mode > 2) return DGFV_ERR_ARG;
    c->launch_mode = mode;
    c->graph_valid = false;
    return DGFV_OK;
}

int dgfv_set_fv_variant(dgfv_ctx* c, int variant) {
    if (!c || variant < 0 || variant > 3) return DGFV_ERR_ARG;
    c->fv_variant = variant;
    c->graph_valid = false;
    return DGFV_OK;
}

int dgfv_autotune(dgfv_ctx* c, int* per_tile_out, void* stream) {
    const NvtxRange nvtx_range("dgfv_autotune");
    if (!c) return DGFV_ERR_ARG;
    TRY(check_dev(c));
    if (!c->state_valid) return fail(c, DGFV_ERR_STATE, "autotune before set_state");
    cudaStream_t s = (cudaStream_t)stream;
    const Params P0 = params(c);
    const Faces F{c->d_faceL, c->d_faceR, c->d_faceD};
    // face values and lifting values of the current state, read by the volume kernel
    launch_prolong(c->nk, P0, c->all.view(), c->all.ntiles, c->d_U, s);
    if (c->n_fv_elems) launch_fv(c->nk, P0, c->fvt.view(), c->fvt.ntiles, c->d_U, s, false, c->fv_variant);
    if (c->ph.viscous) launch_face_lift(c->nk, P0, F, c->lift.d, c->lift.count, s);
    CK(cudaStreamSynchronize(s));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    // launch variant first, on the whole volume launch with the default tiles
    {
        for (int n = 0; n <= MAXDG; ++n) c->vol_per_tile[n] = 0;
        TRY(apply_layout(c));
        const Params P = params(c);
        double best_ms = 1e300;
        int best = 0;
        for (int var = 0; var < (c->opts.split_form ? 0 : 4); ++var) {  // the split kernel has one variant
            launch_dg_volume(c->nk, P, c->dg.view(), c->dg.ntiles, c->dg.smem, c->d_U, s, var);  // warm
            CK(cudaEventRecord(e0, s));
            for (int r = 0; r < 3; ++r) launch_dg_volume(c->nk, P, c->dg.view(), c->dg.ntiles, c->dg.smem, c->d_U, s, var);
            CK(cudaEventRecord(e1, s));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best_ms) {
                best_ms = ms;
                best = var;
            }
        }
        c->vol_variant = best;
    }
    int best_all[MAXDG + 1] = {};
    for (int n = 1; n <= MAXDG; ++n) {
        int cnt = 0;
        for (int e = 0; e < c->n_elem; ++e) cnt += (!c->fv[e] && c->npts[e] == n);
        if (cnt == 0) continue;
        double best_ms = 1e300;
        int best = 0, last = -1;
        for (int nodes : {64, 128, 256, 512, 1024, 2048}) {
            const int per = std::max(1, nodes / (n * n * n));
            if (per == last) continue;
            last = per;
            if (per > 1 && per * n * n * n > 2048) continue;
            if (vol_smem(c, n, per) > 200 * 1024) continue;
            c->vol_per_tile[n] = per;
            TileSet& t = c->dg;
            make_tiles(c, t, [&](int e) { return !c->fv[e] && c->npts[e] == n; }, [&](int) { return per; });
            TRY(upload_tiles(c, t));
            const size_t sm = vol_smem(c, n, per);
            const Params P = params(c);
            launch_volume(c, P, t.view(), t.ntiles, sm, c->d_U, s, c->vol_variant);  // warm
            CK(cudaEventRecord(e0, s));
            for (int r = 0; r < 3; ++r) launch_volume(c, P, t.view(), t.ntiles, sm, c->d_U, s, c->vol_variant);
            CK(cudaEventRecord(e1, s));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best_ms) {
                best_ms = ms;
                best = per;
            }
        }
        best_all[n] = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int n = 1; n <= MAXDG; ++n) {
        c->vol_per_tile[n] = best_all[n];
        if (per_tile_out) per_tile_out[n] = best_all[n];
    }
    if (per_tile_out) per_tile_out[0] = c->vol_variant;
    TRY(apply_layout(c));
    return DGFV_OK;
}

int dgfv_sync_status(dgfv_ctx* c, void* stream) {
    if (!c) return DGFV_ERR_ARG;
    TRY(check_dev(c));
    return read_status(c, (cudaStream_t)stream);
}

int64_t dgfv_bank_entry(dgfv_ctx* c, int which, int N, int M, double* out, int64_t cap) {
    if (!c || !out) return DGFV_ERR_ARG;
    if (N < c->N_min || N > c->N_max) return DGFV_ERR_ARG;
    const int n = N + 1, m = M + 1;
    std::vector<double> v;
    try {
        const int kind = c->opts.nodes;
        Bank1D b = make_bank(n, kind);
        switch (which) {
            case 0: v = b.x; break;
            case 1: v = b.w; break;
            case 2: v = b.Dhat; break;
            case 3: v = b.lm; break;
            case 4: v = b.lp; break;
            case 5:
                if (M < c->N_min || M > c->N_max) return DGFV_ERR_ARG;
                v = make_vmap(n, m, kind);
                break;
            case 6:  // V^{DG->FV} to the context's sub-cell count, or to M sub-cells (M >= 1)
                v = make_dg2fv(n, M >= 1 ? M : c->nfv, kind);
                break;
            case 7: {  // V^{FV->DG} from the context's sub-cell count, or from M sub-cells
                const int nf = M >= 1 ? M : c->nfv;
                v = nf >= n ? make_fv2dg(n, nf, kind) : make_fv2dg_l2(n, nf, kind);
                break;
            }
            case 14:  // sub-cell overlaps from N+1 to M sub-cells per direction
                if (M < 1 || M > MAXP) return DGFV_ERR_ARG;
                v = make_fv_overlap(n, M);
                break;
            case 8: v = b.vinv; break;
            case 9: v = b.D; break;
            case 10:  // mortar maps of half M (0 or 1), Sec. 3.2.3
            case 11:
                if (M < 0 || M > 1) return DGFV_ERR_ARG;
                v = make_mortar(n, M, which == 11, kind);
                break;
            case 12:
            case 13:
                if (M < 0 || M > 1) return DGFV_ERR_ARG;
                v = make_mortar_fv(c->nfv, M, which == 13);
                break;
            default: return DGFV_ERR_ARG;
        }
    } catch (...) {
        return DGFV_ERR_ARG;
    }
    if ((int64_t)v.size() > cap) return DGFV_ERR_ARG;
    std::copy(v.begin(), v.end(), out);
    return (int64_t)v.size();
}

int dgfv_pp_limit(dgfv_ctx* c, double* d_U, int64_t* changed, void* stream) {
    if (!c || !d_U) return DGFV_ERR_ARG;
    TRY(check_dev(c));
    cudaStream_t s = (cudaStream_t)stream;
    const double eps = c->opts.pp_eps > 0.0 ? c->opts.pp_eps : 1e-10;
    unsigned long long* cnt = c->d_pp_count + 1;  // scratch counter of this call
    CK(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
    launch_pp_limit(c->nk, params(c), c->dg.d_items, (int)c->dg.items.size(), d_U, eps, cnt, false, s);
    CK(cudaGetLastError());
    if (changed) {
        unsigned long long h = 0;
        CK(cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        *changed = (int64_t)h;
    }
    return DGFV_OK;
}

int dgfv_pp_count(dgfv_ctx* c, int64_t* count, int reset, void* stream) {
    if (!c || !count) return DGFV_ERR_ARG;
    TRY(check_dev(c));
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long h = 0;
    CK(cudaMemcpyAsync(&h, c->d_pp_count, sizeof(h), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *count = (int64_t)h;
    if (reset) CK(cudaMemsetAsync(c->d_pp_count, 0, sizeof(unsigned long long), s));
    return DGFV_OK;
}

double dgfv_probe_dfma(int iters, void* stream) { return probe_dfma(iters, (cudaStream_t)stream); }

double dgfv_probe_dmma(int iters, void* stream) { return probe_dmma(iters, (cudaStream_t)stream); }

}  // extern "C"
