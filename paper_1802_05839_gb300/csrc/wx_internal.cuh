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
// Resident fields are stored as interleaved (T, q) cells, x fastest:
//   cell[k][jp][ip],  jp = j + 1 in [0, ny+2),  ip = i + kGhostX in [0, P).
// Row jp = 0 and jp = ny+1 and columns ip = kGhostX-1 and ip = kGhostX+nx
// are the periodic ghost ring (copies of the opposite interior edge).  The
// interior starts kGhostX cells into each row so that a warp's 32-cell row
// segment starts on a 128-byte boundary in FP32.
constexpr int kGhostX = 16;
constexpr int kTileX = 32;       // columns per tile in x (one warp)
constexpr int kBoxX = 36;        // TMA box width in cells: 32 + halo, even start
constexpr int kTab = 8;          // per-level table entries

// per-level table entries (one row of kTab values per level k)
enum { TAB_WU = 0, TAB_WD, TAB_AHAT, TAB_CHAT, TAB_WTAU, TAB_WH, TAB_DZ, TAB_PAD };

// device status word bits
enum : unsigned { ST_NONFINITE = 1u, ST_TIMEOUT = 2u, ST_BADARG = 4u };

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

template <typename T> struct StepArgs {
    typename Vec2<T>::type *out;  // new state (interleaved cells)
    const T *U, *V;               // face winds [ny][nx]
    const T *kmult;               // [ny][nx] or nullptr
    const T *tab;                 // [nz][kTab]
    unsigned *status;
    double *partials;             // [gridDim.x*gridDim.y][2] (sums)
    int nx, ny, nz, P, R;
    T dth, dh;                    // dt/h, dt*kappa_h/h^2
    int advection;
};

// A step-kernel configuration: rows per tile, pipeline stages and planes
// per stage.  Chosen per grid by the launcher (or by the autotuner).
struct StepCfg {
    int ty = 4, stages = 6, kb = 2;
};

struct SmemPlan {
    int tab_off, ring_off, state_off, bar_off, total, stage_bytes;
};

__host__ __device__ inline int align_up(int x, int a) { return (x + a - 1) / a * a; }

__host__ __device__ inline SmemPlan plan_smem(int nz, int ty, int stages, int kb, int cell_bytes,
                                              int t_bytes, int narr) {
    SmemPlan p;
    const int nt = kTileX * ty;
    p.tab_off = 0;
    p.ring_off = align_up(nz * kTab * t_bytes, 128);
    p.stage_bytes = align_up(kb * (ty + 2) * kBoxX * cell_bytes, 128);
    p.state_off = align_up(p.ring_off + stages * p.stage_bytes, 128);
    p.bar_off = align_up(p.state_off + narr * nz * nt * t_bytes, 16);
    p.total = p.bar_off + stages * 8 + 16;
    return p;
}

}  // namespace wx

// ------------------------------------------------------------- context
struct wx_ctx {
    int nx = 0, ny = 0, nz = 0, dtype = 0;
    int P = 0, R = 0;            // row pitch (cells) and rows per plane
    size_t plane_cells = 0, field_cells = 0;
    int cell_bytes = 0, t_bytes = 0;
    int device = 0, num_sms = 0;

    void *fld[2] = {nullptr, nullptr};
    int cur = 0;
    CUtensorMap tmap[2];

    void *U = nullptr, *V = nullptr, *kmult = nullptr, *tab = nullptr;
    double *d_lev = nullptr;     // FP64 dz, kappa_lev, alpha [3][nz]
    double *staging = nullptr;   // FP64 [2][nz][ny][nx] for load / read
    unsigned *d_status = nullptr;
    double *partials = nullptr;
    size_t partials_cap = 0;
    double *sums_ring = nullptr;
    int sums_cap = 4096;
    long sums_count = 0;

    // parameters (host copies)
    double dt = 0, h = 0, kappa_h = 0, S0 = 0, q_ref = 0, dd_threshold = 1.1;
    unsigned flags = 0;
    std::vector<double> dz, kappa_lev, alpha, kmult_h, U_h, V_h;
    bool params_set = false, fields_loaded = false, cfl_ok = false;

    // WX_MIXED: columns whose elimination runs in FP64
    int *flag_list = nullptr;    // [n_flag] column index j*nx+i
    double *flag_fac = nullptr;  // [nz][n_flag][2] FP64 elimination factors
    unsigned char *flag_mask = nullptr;  // [ny*nx]
    float *flag_rhs = nullptr;   // [nz][n_flag] T* of flagged columns
    long n_flag = 0;

    wx::StepCfg cfg;
    bool cfg_forced = false;
    cudaStream_t last_stream = nullptr;
    long last_launches = 0;
    std::string err;
};

namespace wx {

// launchers implemented in wx_step.cu
int launch_tables(wx_ctx *c, cudaStream_t s);
int launch_pack(wx_ctx *c, const double *T, const double *q, void *dst, cudaStream_t s);
int launch_unpack(wx_ctx *c, const void *src, double *T, double *q, cudaStream_t s);
int launch_convert(wx_ctx *c, const double *src, void *dst, size_t n, cudaStream_t s);
int launch_step(wx_ctx *c, cudaStream_t s, long *launches);
int launch_columns(wx_ctx *c, const void *Ts, const void *qs, const void *km, void *Tout, void *tend,
                   long ncol, cudaStream_t s);
StepCfg default_cfg(const wx_ctx *c);
bool cfg_fits(const wx_ctx *c, const StepCfg &cfg, int *smem_bytes);
int encode_tmap(wx_ctx *c, int which, int ty, int kb);

}  // namespace wx
