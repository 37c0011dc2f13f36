// wx_internal.cuh -- library-internal types shared by the .cu files of
// libwx.so (context layout, kernel argument blocks, launch helpers).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/wx.h"

namespace wx {

// ---------------------------------------------------------------- layout
// Resident fields are stored plane by plane, x fastest:
//   fld[((k*2 + f)*R + jp)*P + ip],  f = 0 (T) or 1 (q),
//   jp = j + 1 in [0, R = ny+2),  ip = i + kGhostX in [0, P).
// Rows jp = 0 and jp = ny+1 and columns ip = kGhostX-1 and ip = kGhostX+nx
// form the periodic ghost ring (copies of the opposite interior edge).  The
// interior starts kGhostX cells into each row so that a warp's 64-column row
// segment starts on a 64-byte boundary in FP32.
constexpr int kGhostX = 16;
constexpr int kTileX = 64;     // columns per tile in x (one warp, 2 per lane)
constexpr int kBoxX = 72;      // TMA box width: 64 + halo, start a multiple of 4
constexpr int kBoxX0 = 4;      // interior column 0 of a tile sits at box x = 4
constexpr int kTabRec = 6;     // 4-value records per level in the table

// Per-level table: kTabRec record arrays of nz records, record-major:
//  A[k] = {wU, wU, wD, wD}          explicit vertical weights, paired for f32x2
//  B[k] = {-(wU+wD), -(wU+wD), wt2, wt2}  centre correction; optical depth per
//                                   unit q in log2 units, alpha dz log2(e)/q_ref
//  C[k] = {wH, wH, -c_k, -c_k}      dt S0/dz_k; minus the super-diagonal of the
//                                   kappa_mult = 1 column
//  D[k] = {1/m_k, 1/m_k, e_k, e_k}  that column's top-down elimination:
//                                   m_k = b_k - c_k e_{k+1}, e_k = a_k/m_k
//  E[k] = {ahat_k, chat_k, dz_k, 0} sub/super-diagonal per unit kappa_mult
//  F[k] = {-e_k, -e_k, dz_k, dz_k}  back substitution and sums
// with wU = dt kappa_h/(dz_k g_{k+1/2}) (0 at the top), wD likewise below.
enum { REC_A = 0, REC_B = 1, REC_C = 2, REC_D = 3, REC_E = 4, REC_F = 5 };

template <typename T> struct alignas(4 * sizeof(T)) Q4 { T x, y, z, w; };

// device status word bits
enum : unsigned { ST_NONFINITE = 1u, ST_TIMEOUT = 2u, ST_BADARG = 4u, ST_BOUNDS = 8u };

// Range checks of the bounds-checked build (compiled with WX_BOUNDS_CHECK,
// libwx_bounds.so): an access whose element offset is outside its buffer is
// skipped and reported through the status word (ST_BOUNDS), never trapped.
// In the release build every check is the constant true.
__device__ __forceinline__ bool bounds_ok(long long off, long long n, unsigned *status) {
    if (off >= 0 && off < n) return true;
    atomicOr(status, ST_BOUNDS);
    return false;
}
#ifdef WX_BOUNDS_CHECK
#define WX_IN(off, n, status) ::wx::bounds_ok((long long)(off), (long long)(n), (status))
#else
#define WX_IN(off, n, status) true
#endif

// One level of the Thomas forward sweep of a column's implicit vertical
// diffusion, (I - dt L_v) x = r with zero-flux ends, in a form in which
// nothing cancels.  The sub- and super-diagonals are a_k = -na_k <= 0 and
// c_k = -nc_k <= 0 and the diagonal b_k = 1 + na_k + nc_k, so the textbook
// pivot m_k = b_k - a_k c'_{k-1} equals 1 + nc_k + na_k g_{k-1} with
// g_k = 1 + c'_k = (1 + na_k g_{k-1}) / m_k: sums of nonnegative terms only.
// The textbook form subtracts two numbers of size ~na_k when the column is
// near-singular (na, nc >> 1) and loses that many digits in FP32.
template <typename T> struct ThomasSweep {
    T g = T(0), d = T(0);  // g_{k-1} and d'_{k-1}
    // advances to level k (na_0 = 0 at the bottom); returns c'_k, d holds d'_k
    __device__ __forceinline__ T level(T na, T nc, T r) {
        const T m = fma(na, g, T(1) + nc);
        const T inv = T(1) / m;
        g = fma(na, g, T(1)) * inv;
        d = fma(na, d, r) * inv;
        return -nc * inv;
    }
};

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

template <typename T> struct StepArgs {
    T *out;                       // new state (planar fields)
    const T *U, *V;               // face winds [ny][nx]
    const T *kmult;               // [ny][nx] or nullptr
    const Q4<T> *tab;             // [kTabRec][nz]
    unsigned *status;
    double *partials;             // [tiles][2] (sums)
    int nx, ny, nz, P, R;
    T dth, dh;                    // dt/h, dt*kappa_h/h^2
    int advection;
    // WX_MIXED: listed columns park T* and dt*H in side[k][0][f], side[k][1][f]
    const int *flag_idx;          // [ny][nx]: index f of a listed column, else -1
    float *side;                  // [nz][2][n_list]
    long n_list;
    // sub-domain of a decomposed grid: the west-face winds of column 0
    // ([ny]) and the south-face winds of row 0 ([nx]) come from the
    // neighbours (nullptr: periodic within this grid)
    const T *Uw0, *Vs0;
    long long out_n;              // elements of `out` (bounds-checked build)
};

// One member of a (possibly single-member) batch stepped by one launch:
// its input-state descriptor, its arguments and the first index of its tiles
// in the combined (member, tile) work list.
constexpr int kMaxMembers = 16;
template <typename T> struct alignas(64) Member {
    CUtensorMap tin;
    CUtensorMap tbase;  // RK3 stage launches: the base state's interior boxes
    StepArgs<T> a;
    long tile0;
    int gx, gy;
};
template <typename T> struct Members {
    Member<T> m[kMaxMembers];
    int n;
    int nz_max;
    long total;          // work items (tiles of all members)
    unsigned *status;
};

// A step-kernel configuration: rows per tile, TMA ring stages (2 planes
// each), resident CTAs per SM and L2 prefetch distance in stages.  Chosen by
// a heuristic at create time or set by the autotuner.
struct StepCfg {
    int ty = 2, stages = 4, kb = 2, ctas_per_sm = 4, prefetch = 8;
};

struct SmemPlan {
    int tab_off, ring_off, state_off, bar_off, total, stage_bytes;
};

__host__ __device__ inline int align_up(int x, int a) { return (x + a - 1) / a * a; }

// TMEM column state of the FP32 step kernel: every consumer lane keeps F_k
// of its two columns (2 nz <= 128 words) in its own TMEM lane; warps w,
// w + 4 and w + 8 share a lane quarter and take 128 columns each, so a CTA
// allocates 128 (4 consumer warps), 256 (8) or all 512 (12) columns.
constexpr int kTmemMaxNz = 64;
__host__ __device__ constexpr uint32_t kTmemCols(int ty) { return ty > 8 ? 512u : (ty > 4 ? 256u : 128u); }

// Shared-memory plan of the step kernel: per-level table, TMA ring of
// `stages` slots (kb planes x 2 fields x (ty+2) rows x kBoxX), per-thread
// column state (F_k of the lane's two columns, plus their e_k for per-column
// kappa; none when it lives in TMEM), then full/empty mbarriers and the
// TMEM address.
__host__ __device__ inline int box_bytes(int ty, int kb, int t_bytes) {
    return align_up(kb * 2 * (ty + 2) * kBoxX * t_bytes, 128);
}
// A stage slot of an RK3 stage launch also holds the base state phi^n of
// the tile's interior (kb planes x 2 fields x ty rows x kTileX), after the
// halo box.
__host__ __device__ inline int base_box_bytes(int ty, int kb, int t_bytes) {
    return align_up(kb * 2 * ty * kTileX * t_bytes, 128);
}
__host__ __device__ inline SmemPlan plan_smem(int nz, int ty, int stages, int kb, int t_bytes,
                                              bool per_col, bool tmem = false, bool rk_base = false) {
    SmemPlan p;
    const int nt = 32 * ty;
    p.tab_off = 0;
    p.ring_off = align_up(kTabRec * nz * 4 * t_bytes, 128);
    p.stage_bytes = box_bytes(ty, kb, t_bytes) + (rk_base ? base_box_bytes(ty, kb, t_bytes) : 0);
    p.state_off = align_up(p.ring_off + stages * p.stage_bytes, 128);
    const int state = tmem ? 0 : nz * nt * 2 * t_bytes * (per_col ? 2 : 1);
    p.bar_off = align_up(p.state_off + state, 16);
    p.total = p.bar_off + 2 * stages * 8 + 16;
    return p;
}

}  // namespace wx

// ------------------------------------------------------------- context
struct wx_ctx {
    int nx = 0, ny = 0, nz = 0, dtype = 0;
    int P = 0, R = 0;            // row pitch (cells) and rows per plane
    size_t plane_cells = 0, field_cells = 0;  // one (k, f) plane; whole array
    int cell_bytes = 0, t_bytes = 0;
    int device = 0, num_sms = 0;

    void *fld[3] = {nullptr, nullptr, nullptr};  // ping-pong + the RK3 stage buffer
    int cur = 0;
    CUtensorMap tmap[3];
    // WX_RK3: tables of the three stage steps dt/3, dt/2, dt; while a stage
    // runs, the batch launcher reads buffer stage_in, writes stage_out with
    // step stage_dt and table stage_tab, and leaves `cur` alone
    void *tab_rk = nullptr;
    int stage_in = -1, stage_out = -1;
    double stage_dt = 0;
    const void *stage_tab = nullptr;
    // a stage launch that writes phi^n + (E - phi_s) itself: the base buffer
    // phi^n and its interior-box descriptor (-1: the stage writes E)
    int stage_base = -1;
    CUtensorMap tmap_rkbase;

    void *U = nullptr, *V = nullptr, *kmult = nullptr, *tab = nullptr;
    double *d_lev = nullptr;     // FP64 dz, kappa_lev, alpha [3][nz]
    double *staging = nullptr;   // FP64 [2][nz][ny][nx] for load / read
    unsigned *d_status = nullptr;
    double *partials = nullptr;
    size_t partials_cap = 0;
    double *sums_ring = nullptr;
    double *fin_park = nullptr;     // [64][2] per-block results of the sums reduction
    unsigned *fin_ticket = nullptr; // arrival counter of the sums reduction (self-resetting)
    int sums_cap = 4096;
    long long *d_sums_count = nullptr;  // steps recorded since the last load (device)

    // parameters (host copies)
    double dt = 0, h = 0, kappa_h = 0, S0 = 0, q_ref = 0, dd_threshold = 1.1;
    unsigned flags = 0;
    std::vector<double> dz, kappa_lev, alpha, kmult_h, U_h, V_h;
    bool params_set = false, fields_loaded = false, cfl_ok = false;

    // WX_MIXED: columns whose elimination runs in FP64
    int *flag_list = nullptr;    // [n_flag] column index j*nx+i
    int *flag_idx = nullptr;     // [ny*nx] f or -1
    double *flag_fac = nullptr;  // [nz][n_list][2] FP64 (1/m_k, c_k/m_k) from the top
    float *flag_e = nullptr;     // [nz][n_list] e_k for the FP32 back substitution
    float *flag_side = nullptr;  // [nz][2][n_list] T* and dt*H parked by the step kernel
    double *flag_corr = nullptr; // [n_flag] energy correction of the FP64 solve (sums)
    long n_flag = 0;             // columns solved in FP64 (first in the list)
    long n_list = 0;             // all listed columns (kappa_mult != 1)
    bool fixup_carveout = false; // the side kernel's shared-memory carveout is set on this device

    // WX_SURROGATE: the attached network and this grid's activation buffers
    struct wx_mlp *sur = nullptr;
    double sur_tol = 2e-2;
    long sur_rows = 0;            // nx*ny rounded up to 128
    void *sur_X = nullptr, *sur_H[2] = {nullptr, nullptr};
    float *sur_Y = nullptr, *sur_lev = nullptr;  // [rows][128]; [2][nz] kappa_lev, alpha dz
    unsigned long long *sur_nfb = nullptr;       // [0] fallbacks of the last network step, [1] probe rejections
    unsigned sur_gen = ~0u;       // generation sur_lev was built for
    // acceptance policy (wx_set_surrogate_policy): the network runs while
    // its measured acceptance is at least sur_min_accept; otherwise steps
    // are exact fused steps, and every sur_probe_every steps the network is
    // probed on sur_probe_rows rows of the state.  Decisions use the counts
    // of the step two before (read back through pinned memory and events).
    double sur_min_accept = 0.0;
    int sur_probe_every = 8, sur_probe_rows = 16;
    int sur_mode = 0;             // 0: network steps, 1: exact steps
    bool sur_last_exact = false;  // the last step ran no network
    long long sur_step = 0, sur_next_probe = 0;
    int sur_probe_row0 = 0;
    static constexpr int kSurRing = 8;
    struct SurRead {
        long long step = -1;
        long ncols = 0;
        int slot = 0;
    };
    std::vector<SurRead> sur_reads;          // outstanding counts, oldest first
    unsigned long long *sur_host = nullptr;  // pinned [kSurRing]
    cudaEvent_t sur_ev[kSurRing] = {};
    int sur_slot = 0;

    // sub-domain of a wx_dom: neighbours' face winds at the west column and
    // the south row (device, storage type; host FP64 copies for the CFL
    // check)
    void *Uw0 = nullptr, *Vs0 = nullptr;
    std::vector<double> Uw0_h, Vs0_h;

    wx::StepCfg cfg;
    bool cfg_forced = false;
    cudaStream_t last_stream = nullptr;
    long last_launches = 0;
    unsigned generation = 0;     // bumped by every change a captured graph would bake in
    std::string err;
};

namespace wx {

// launchers implemented in wx_step.cu
int launch_tables(wx_ctx *c, cudaStream_t s);
int launch_tables_dt(wx_ctx *c, double dt, void *dst, cudaStream_t s);
int launch_rk3_step(wx_ctx *c, cudaStream_t s, long *launches);
int launch_pack(wx_ctx *c, const double *T, const double *q, void *dst, cudaStream_t s);
int launch_unpack(wx_ctx *c, const void *src, double *T, double *q, cudaStream_t s);
int launch_pack_f32(wx_ctx *c, const float *T, const float *q, void *dst, cudaStream_t s);
int launch_unpack_f32(wx_ctx *c, const void *src, float *T, float *q, cudaStream_t s);
int launch_convert(wx_ctx *c, const double *src, void *dst, size_t n, cudaStream_t s);
int launch_step(wx_ctx *c, cudaStream_t s, long *launches);
int launch_batch(wx_ctx *const *members, int n, const StepCfg &cfg, unsigned *status, cudaStream_t s,
                 long *launches, std::string &err);
int launch_columns(wx_ctx *c, const void *Ts, const void *qs, const void *km, void *Tout, void *tend,
                   long ncol, cudaStream_t s);
StepCfg default_cfg(const wx_ctx *c);
int setup_mixed(wx_ctx *c, const double *km64);
// The side solve of the listed columns after a step into fld[dst] (WX_MIXED,
// or WX_F32 with kappa_mult); with sums, their energy corrections.
int launch_mixed_fixup(wx_ctx *c, int dst, bool sums, cudaStream_t s);
bool cfg_fits(const wx_ctx *c, const StepCfg &cfg, int *smem_bytes);
int encode_tmap(wx_ctx *c, int which, int ty, int kb);
// descriptor of the interior boxes (kTileX x ty x 2 x kb) of buffer `which`
int encode_tmap_interior(wx_ctx *c, int which, int ty, int kb, CUtensorMap *out);
int apply_cfg(wx_ctx *c, const StepCfg &g);
int check_cfl(wx_ctx *c);
// WX_SURROGATE (wx_mlp.cu)
int launch_surrogate_step(wx_ctx *c, cudaStream_t s, long *launches);
// one WX_SURROGATE step under the context's acceptance policy
int launch_surrogate_policy_step(wx_ctx *c, cudaStream_t s, long *launches);
// forget the policy's measurements (a new state was loaded)
void reset_surrogate_policy(wx_ctx *c);
void free_surrogate(wx_ctx *c);

}  // namespace wx
