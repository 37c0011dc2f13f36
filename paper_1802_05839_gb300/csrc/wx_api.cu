// wx_api.cu -- the C ABI of libwx.so (declared in include/wx.h): context
// life cycle, parameter validation, resident-field layout, TMA descriptors,
// the step loop and the checkpoint / sums read-back.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "ptx.cuh"
#include "wx_internal.cuh"

using namespace wx;

static thread_local std::string g_create_error;

static int fail(wx_ctx *c, int code, const std::string &msg) {
    if (c)
        c->err = msg;
    else
        g_create_error = msg;
    return code;
}

static int cuda_fail(wx_ctx *c, cudaError_t e, const char *what) {
    return fail(c, WX_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call, what)                                        \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

#define RC(call)                   \
    do {                           \
        int r_ = (call);           \
        if (r_ != WX_OK) return r_; \
    } while (0)

// ------------------------------------------------------------ TMA maps
static PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

namespace wx {
// Describe a resident state as a 4D tensor of T elements {x: P, y: ny+2,
// field: 2, z: nz} (planar T and q planes per level); box = 72 x (ty+2) x 2
// fields x kb planes, x start a multiple of 4 elements (16-byte aligned).
int encode_tmap(wx_ctx *c, int which, int ty, int kb) {
    auto enc = tmap_encoder();
    if (!enc) return fail(c, WX_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint64_t t = (cuuint64_t)c->t_bytes;
    cuuint64_t dims[4] = {(cuuint64_t)c->P, (cuuint64_t)c->R, 2, (cuuint64_t)c->nz};
    cuuint64_t strides[3] = {(cuuint64_t)c->P * t, (cuuint64_t)c->P * c->R * t, 2 * (cuuint64_t)c->P * c->R * t};
    cuuint32_t box[4] = {(cuuint32_t)kBoxX, (cuuint32_t)(ty + 2), 2, (cuuint32_t)kb};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUtensorMapDataType dt =
        c->t_bytes == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    CUresult r = enc(&c->tmap[which], dt, 4, c->fld[which], dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(c, WX_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string(r) + ")");
    return WX_OK;
}

// The same tensor with boxes of a tile's interior: kTileX x ty x 2 fields x
// kb planes, x start kGhostX + kTileX * bx (a multiple of 16 elements).
int encode_tmap_interior(wx_ctx *c, int which, int ty, int kb, CUtensorMap *out) {
    auto enc = tmap_encoder();
    if (!enc) return fail(c, WX_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint64_t t = (cuuint64_t)c->t_bytes;
    cuuint64_t dims[4] = {(cuuint64_t)c->P, (cuuint64_t)c->R, 2, (cuuint64_t)c->nz};
    cuuint64_t strides[3] = {(cuuint64_t)c->P * t, (cuuint64_t)c->P * c->R * t, 2 * (cuuint64_t)c->P * c->R * t};
    cuuint32_t box[4] = {(cuuint32_t)kTileX, (cuuint32_t)ty, 2, (cuuint32_t)kb};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUtensorMapDataType dt =
        c->t_bytes == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    CUresult r = enc(out, dt, 4, c->fld[which], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(c, WX_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string(r) + ")");
    return WX_OK;
}
}  // namespace wx

namespace wx {
int apply_cfg(wx_ctx *c, const StepCfg &g) {
    c->cfg = g;
    ++c->generation;
    RC(encode_tmap(c, 0, g.ty, g.kb));
    RC(encode_tmap(c, 1, g.ty, g.kb));
    if (c->fld[2]) RC(encode_tmap(c, 2, g.ty, g.kb));
    return WX_OK;
}
}  // namespace wx

// ------------------------------------------------------------ life cycle
extern "C" int wx_create(int nx, int ny, int nz, int dtype, wx_ctx **out) {
    if (!out) return fail(nullptr, WX_EINVAL, "wx_create: out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return fail(nullptr, WX_EINVAL, "wx_create: sizes must be >= 1");
    if (dtype != WX_F32 && dtype != WX_F64 && dtype != WX_MIXED)
        return fail(nullptr, WX_EINVAL, "wx_create: unknown dtype");
    if (nz > 256) return fail(nullptr, WX_EUNSUPPORTED, "wx_create: nz > 256 is not supported");
    if ((long)nx > (1L << 24) || ny > 65535)
        return fail(nullptr, WX_EUNSUPPORTED, "wx_create: nx must be < 2^24 and ny <= 65535");
    wx_ctx *c = new (std::nothrow) wx_ctx();
    if (!c) return fail(nullptr, WX_ENOMEM, "wx_create: host allocation failed");
    c->nx = nx;
    c->ny = ny;
    c->nz = nz;
    c->dtype = dtype;
    c->t_bytes = dtype == WX_F64 ? 8 : 4;
    c->cell_bytes = 2 * c->t_bytes;
    c->P = align_up(kGhostX + nx + 1, 16);
    c->R = ny + 2;
    c->plane_cells = (size_t)c->P * c->R;
    c->field_cells = c->plane_cells * nz;

    auto bail = [&](int code) {
        g_create_error = c->err;
        wx_destroy(c);
        return code;
    };
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        c->err = "wx_create: no CUDA device";
        return bail(WX_ECUDA);
    }
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    const size_t fbytes = c->field_cells * c->cell_bytes;
    const size_t cols = (size_t)nx * ny;
    const size_t nblk_max = (size_t)((nx + kTileX - 1) / kTileX) * ny;
    struct {
        void **p;
        size_t n;
    } allocs[] = {{&c->fld[0], fbytes},
                  {&c->fld[1], fbytes},
                  {&c->U, cols * c->t_bytes},
                  {&c->V, cols * c->t_bytes},
                  {&c->tab, (size_t)nz * kTabRec * 4 * c->t_bytes},
                  {(void **)&c->d_lev, 3 * (size_t)nz * sizeof(double)},
                  {(void **)&c->d_status, sizeof(unsigned)},
                  {(void **)&c->partials, 2 * nblk_max * sizeof(double)},
                  {(void **)&c->sums_ring, 2 * (size_t)c->sums_cap * sizeof(double)},
                  {(void **)&c->fin_park, 2 * 64 * sizeof(double)},
                  {(void **)&c->fin_ticket, sizeof(unsigned)},
                  {(void **)&c->d_sums_count, sizeof(long long)}};
    for (auto &a : allocs) {
        cudaError_t e = cudaMalloc(a.p, a.n);
        if (e != cudaSuccess) {
            cudaGetLastError();
            c->err = std::string("wx_create: device allocation failed: ") + cudaGetErrorString(e);
            return bail(WX_ENOMEM);
        }
    }
    c->partials_cap = nblk_max;
    if (cudaMemset(c->fld[0], 0, fbytes) != cudaSuccess || cudaMemset(c->fld[1], 0, fbytes) != cudaSuccess ||
        cudaMemset(c->d_status, 0, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(c->fin_ticket, 0, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(c->d_sums_count, 0, sizeof(long long)) != cudaSuccess ||
        cudaMemset(c->U, 0, cols * c->t_bytes) != cudaSuccess ||
        cudaMemset(c->V, 0, cols * c->t_bytes) != cudaSuccess) {
        c->err = "wx_create: cudaMemset failed";
        return bail(WX_ECUDA);
    }
    int rc = apply_cfg(c, default_cfg(c));
    if (rc != WX_OK) return bail(rc);
    *out = c;
    return WX_OK;
}

extern "C" void wx_destroy(wx_ctx *c) {
    if (!c) return;
    free_surrogate(c);
    void *ptrs[] = {c->fld[0], c->fld[1], c->fld[2], c->tab_rk, c->U, c->V, c->kmult, c->tab,
                    c->d_lev,  c->staging, c->d_status, c->partials, c->sums_ring, c->flag_list,
                    c->flag_idx, c->flag_fac, c->flag_e, c->flag_side, c->flag_corr,
                    c->fin_park, c->fin_ticket, c->d_sums_count, c->Uw0, c->Vs0};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete c;
}

extern "C" const char *wx_last_error(const wx_ctx *c) {
    return c ? c->err.c_str() : g_create_error.c_str();
}

extern "C" int wx_info(const wx_ctx *c, int *nx, int *ny, int *nz, int *dtype, long *pitch, long *bytes) {
    if (!c) return WX_EINVAL;
    if (nx) *nx = c->nx;
    if (ny) *ny = c->ny;
    if (nz) *nz = c->nz;
    if (dtype) *dtype = c->dtype;
    if (pitch) *pitch = c->P;
    if (bytes) *bytes = (long)(2 * c->field_cells * c->cell_bytes);
    return WX_OK;
}

extern "C" long wx_last_launches(const wx_ctx *c) { return c ? c->last_launches : -1; }

extern "C" int wx_flagged_columns(const wx_ctx *c, long *n) {
    if (!c || !n) return WX_EINVAL;
    *n = c->n_flag;
    return WX_OK;
}

extern "C" int wx_set_step_config(wx_ctx *c, int ty, int kb, int stages, int ctas_per_sm, int prefetch) {
    if (!c) return WX_EINVAL;
    if (!(ty == 1 || ty == 2 || ty == 4 || ty == 8 || ty == 12) || !(kb == 2 || kb == 4) || stages < 3 ||
        stages > 16 || ctas_per_sm < 1 || prefetch < 0 || prefetch > 64)
        return fail(c, WX_EINVAL,
                    "wx_set_step_config: ty in {1,2,4,8,12}, kb in {2,4}, stages 3..16, ctas >= 1, prefetch 0..64");
    if (ty == 1 && kb == 4) return fail(c, WX_EUNSUPPORTED, "wx_set_step_config: ty = 1 with kb = 4 is not built");
    StepCfg g;
    g.ty = ty;
    g.stages = stages;
    g.kb = kb;
    g.ctas_per_sm = ctas_per_sm;
    g.prefetch = prefetch;
    if (!cfg_fits(c, g, nullptr)) return fail(c, WX_EUNSUPPORTED, "wx_set_step_config: shared memory does not fit");
    RC(apply_cfg(c, g));
    c->cfg_forced = true;
    return WX_OK;
}

extern "C" int wx_get_step_config(const wx_ctx *c, int *ty, int *kb, int *stages, int *ctas, int *prefetch,
                                  int *smem) {
    if (!c) return WX_EINVAL;
    if (ty) *ty = c->cfg.ty;
    if (kb) *kb = c->cfg.kb;
    if (stages) *stages = c->cfg.stages;
    if (ctas) *ctas = c->cfg.ctas_per_sm;
    if (prefetch) *prefetch = c->cfg.prefetch;
    if (smem) cfg_fits(c, c->cfg, smem);
    return WX_OK;
}

// ------------------------------------------------------------ parameters
static bool finite_pos(double x) { return std::isfinite(x) && x > 0; }
static bool finite_nonneg(double x) { return std::isfinite(x) && x >= 0; }

extern "C" int wx_set_params(wx_ctx *c, const wx_params *p) {
    if (!c) return WX_EINVAL;
    if (!p) return fail(c, WX_EINVAL, "wx_set_params: params is NULL");
    if (!finite_pos(p->dt) || !finite_pos(p->h) || !finite_pos(p->q_ref))
        return fail(c, WX_EINVAL, "wx_set_params: dt, h and q_ref must be finite and > 0");
    if (!finite_nonneg(p->kappa_h) || !finite_nonneg(p->S0))
        return fail(c, WX_EINVAL, "wx_set_params: kappa_h and S0 must be finite and >= 0");
    if (!p->dz || !p->kappa_lev || !p->alpha)
        return fail(c, WX_EINVAL, "wx_set_params: dz, kappa_lev and alpha are required");
    if (p->flags & ~(unsigned)(WX_ADVECTION | WX_PHYSICS | WX_SUMS | WX_SURROGATE | WX_RK3))
        return fail(c, WX_EINVAL, "wx_set_params: unknown flag bits");
    if ((p->flags & WX_RK3) && (c->dtype == WX_MIXED || (p->flags & (WX_SUMS | WX_SURROGATE))))
        return fail(c, WX_EUNSUPPORTED, "wx_set_params: WX_RK3 needs WX_F32 or WX_F64 and excludes WX_SUMS, WX_SURROGATE");
    if ((p->flags & WX_SURROGATE) && (c->dtype != WX_F32 || c->nz != 58 || (p->flags & WX_SUMS)))
        return fail(c, WX_EUNSUPPORTED, "wx_set_params: WX_SURROGATE needs WX_F32, nz = 58 and no WX_SUMS");
    const int nz = c->nz;
    if (p->kappa_mult && c->dtype == WX_F64 && plan_smem(nz, 1, 3, 2, 8, true).total > 227 * 1024) {
        // per-column elimination keeps F_k and e_k of every column in shared memory
        int nmax = 1;
        while (plan_smem(nmax + 1, 1, 3, 2, 8, true).total <= 227 * 1024) ++nmax;
        return fail(c, WX_EUNSUPPORTED, "wx_set_params: an FP64 context with kappa_mult takes at most " +
                                            std::to_string(nmax) + " levels");
    }
    for (int k = 0; k < nz; ++k) {
        if (!finite_pos(p->dz[k])) return fail(c, WX_EINVAL, "wx_set_params: dz must be finite and > 0");
        if (!finite_nonneg(p->kappa_lev[k]) || !finite_nonneg(p->alpha[k]))
            return fail(c, WX_EINVAL, "wx_set_params: kappa_lev and alpha must be finite and >= 0");
    }
    const size_t cols = (size_t)c->nx * c->ny;
    if (p->kappa_mult)
        for (size_t e = 0; e < cols; ++e)
            if (!finite_nonneg(p->kappa_mult[e]))
                return fail(c, WX_EINVAL, "wx_set_params: kappa_mult must be finite and >= 0");

    c->dt = p->dt;
    c->h = p->h;
    c->kappa_h = p->kappa_h;
    c->S0 = p->S0;
    c->q_ref = p->q_ref;
    c->dd_threshold = p->dd_threshold > 0 ? p->dd_threshold : 1.1;
    c->flags = p->flags;
    c->dz.assign(p->dz, p->dz + nz);
    c->kappa_lev.assign(p->kappa_lev, p->kappa_lev + nz);
    c->alpha.assign(p->alpha, p->alpha + nz);
    if (p->kappa_mult)
        c->kmult_h.assign(p->kappa_mult, p->kappa_mult + cols);
    else
        c->kmult_h.clear();

    std::vector<double> lev(3 * (size_t)nz);
    std::copy(c->dz.begin(), c->dz.end(), lev.begin());
    std::copy(c->kappa_lev.begin(), c->kappa_lev.end(), lev.begin() + nz);
    std::copy(c->alpha.begin(), c->alpha.end(), lev.begin() + 2 * nz);
    CK(cudaMemcpy(c->d_lev, lev.data(), lev.size() * sizeof(double), cudaMemcpyHostToDevice), "upload levels");
    RC(launch_tables(c, 0));
    if (p->kappa_mult) {
        if (!c->kmult) CK(cudaMalloc(&c->kmult, cols * c->t_bytes), "alloc kappa_mult");
        double *tmp = nullptr;
        CK(cudaMalloc(&tmp, cols * sizeof(double)), "alloc kappa_mult staging");
        cudaError_t e = cudaMemcpy(tmp, p->kappa_mult, cols * sizeof(double), cudaMemcpyHostToDevice);
        int rc = (e == cudaSuccess) ? launch_convert(c, tmp, c->kmult, cols, 0) : cuda_fail(c, e, "upload kappa_mult");
        cudaDeviceSynchronize();
        if (rc == WX_OK) rc = setup_mixed(c, tmp);
        cudaFree(tmp);
        if (rc != WX_OK) return rc;
    } else {
        if (c->kmult) {
            cudaFree(c->kmult);
            c->kmult = nullptr;
        }
        RC(setup_mixed(c, nullptr));
    }
    if (p->flags & WX_RK3) {
        const size_t tbytes = (size_t)nz * kTabRec * 4 * c->t_bytes;
        if (!c->fld[2]) {
            const size_t fbytes = c->field_cells * c->cell_bytes;
            CK(cudaMalloc(&c->fld[2], fbytes), "alloc RK3 stage buffer");
            CK(cudaMemset(c->fld[2], 0, fbytes), "clear RK3 stage buffer");
        }
        if (!c->tab_rk) CK(cudaMalloc(&c->tab_rk, 3 * tbytes), "alloc RK3 tables");
        for (int st = 0; st < 3; ++st)
            RC(launch_tables_dt(c, st == 0 ? c->dt / 3.0 : (st == 1 ? c->dt / 2.0 : c->dt),
                                (char *)c->tab_rk + st * tbytes, 0));
        RC(encode_tmap(c, 2, c->cfg.ty, c->cfg.kb));
    }
    CK(cudaDeviceSynchronize(), "wx_set_params");
    // the kernel variant (and its shared-memory plan) depends on kappa_mult
    if (!c->cfg_forced || !cfg_fits(c, c->cfg, nullptr)) RC(apply_cfg(c, default_cfg(c)));
    ++c->generation;
    c->params_set = true;
    c->cfl_ok = false;
    return WX_OK;
}

// Positivity of the explicit update: every coefficient of phi* as a linear
// combination of old values must be >= 0 (this is what keeps the first-order
// upwind + diffusion scheme monotone).  Checked on the host from the FP64
// parameters and winds.
int wx::check_cfl(wx_ctx *c) {
    if (c->cfl_ok) return WX_OK;
    const int nx = c->nx, ny = c->ny, nz = c->nz;
    const double dh = c->dt * c->kappa_h / (c->h * c->h), dth = c->dt / c->h;
    double wmax = 0;
    for (int k = 0; k < nz; ++k) {
        double w = 0;
        if (k < nz - 1) w += c->dt * c->kappa_h / (c->dz[k] * 0.5 * (c->dz[k] + c->dz[k + 1]));
        if (k > 0) w += c->dt * c->kappa_h / (c->dz[k] * 0.5 * (c->dz[k - 1] + c->dz[k]));
        wmax = std::max(wmax, w);
    }
    double omax = 0;
    if (c->flags & WX_ADVECTION) {
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const double ue = c->U_h[(size_t)j * nx + i];
                const bool hw = i == 0 && !c->Uw0_h.empty(), hs = j == 0 && !c->Vs0_h.empty();
                const double uw = hw ? c->Uw0_h[j] : c->U_h[(size_t)j * nx + (i == 0 ? nx - 1 : i - 1)];
                const double vn = c->V_h[(size_t)j * nx + i];
                const double vs = hs ? c->Vs0_h[i] : c->V_h[(size_t)(j == 0 ? ny - 1 : j - 1) * nx + i];
                if (!std::isfinite(ue) || !std::isfinite(vn))
                    return fail(c, WX_EINVAL, "winds must be finite");
                const double o = std::max(ue, 0.0) - std::min(uw, 0.0) + std::max(vn, 0.0) - std::min(vs, 0.0);
                omax = std::max(omax, o);
            }
    }
    const double worst = 4 * dh + dth * omax + wmax;
    if (worst > 1.0 + 1e-12) {
        char buf[256];
        snprintf(buf, sizeof buf,
                 "positivity bound violated: 4*dt*kappa/h^2 + dt/h*max outflow + max vertical weight = %.6g > 1",
                 worst);
        return fail(c, WX_ECFL, buf);
    }
    c->cfl_ok = true;
    return WX_OK;
}

// ------------------------------------------------------------ state I/O
static int ensure_staging(wx_ctx *c) {
    if (c->staging) return WX_OK;
    const size_t n = 2 * (size_t)c->nx * c->ny * c->nz;
    cudaError_t e = cudaMalloc(&c->staging, n * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->staging = nullptr;
        return fail(c, WX_ENOMEM, "staging allocation failed");
    }
    return WX_OK;
}

extern "C" int wx_load_fields(wx_ctx *c, const double *T, const double *q, const double *U, const double *V,
                              int src_is_device) {
    if (!c) return WX_EINVAL;
    if (!T || !q || !U || !V) return fail(c, WX_EINVAL, "wx_load_fields: NULL array");
    const size_t n = (size_t)c->nx * c->ny * c->nz, cols = (size_t)c->nx * c->ny;
    const double *dT = T, *dq = q, *dU = U, *dV = V;
    c->U_h.resize(cols);
    c->V_h.resize(cols);
    if (!src_is_device) {
        RC(ensure_staging(c));
        double *sT = c->staging, *sq = c->staging + n;
        CK(cudaMemcpy(sT, T, n * sizeof(double), cudaMemcpyHostToDevice), "upload T");
        CK(cudaMemcpy(sq, q, n * sizeof(double), cudaMemcpyHostToDevice), "upload q");
        dT = sT;
        dq = sq;
        std::memcpy(c->U_h.data(), U, cols * sizeof(double));
        std::memcpy(c->V_h.data(), V, cols * sizeof(double));
    } else {
        CK(cudaMemcpy(c->U_h.data(), U, cols * sizeof(double), cudaMemcpyDeviceToHost), "winds to host");
        CK(cudaMemcpy(c->V_h.data(), V, cols * sizeof(double), cudaMemcpyDeviceToHost), "winds to host");
    }
    c->cur = 0;
    RC(launch_pack(c, dT, dq, c->fld[0], 0));
    if (!src_is_device) {
        // winds through the (now free) staging area
        double *sU = c->staging, *sV = c->staging + cols;
        CK(cudaDeviceSynchronize(), "pack");
        CK(cudaMemcpy(sU, U, cols * sizeof(double), cudaMemcpyHostToDevice), "upload U");
        CK(cudaMemcpy(sV, V, cols * sizeof(double), cudaMemcpyHostToDevice), "upload V");
        dU = sU;
        dV = sV;
    }
    RC(launch_convert(c, dU, c->U, cols, 0));
    RC(launch_convert(c, dV, c->V, cols, 0));
    CK(cudaMemset(c->d_sums_count, 0, sizeof(long long)), "reset sums count");
    CK(cudaDeviceSynchronize(), "wx_load_fields");
    reset_surrogate_policy(c);
    ++c->generation;
    c->fields_loaded = true;
    c->cfl_ok = false;
    return WX_OK;
}

extern "C" int wx_read_fields_device(wx_ctx *c, double *T, double *q, void *stream) {
    if (!c) return WX_EINVAL;
    if (!c->fields_loaded) return fail(c, WX_ESTATE, "wx_read_fields: no fields loaded");
    return launch_unpack(c, c->fld[c->cur], T, q, (cudaStream_t)stream);
}

extern "C" int wx_read_fields(wx_ctx *c, double *T, double *q) {
    if (!c) return WX_EINVAL;
    if (!c->fields_loaded) return fail(c, WX_ESTATE, "wx_read_fields: no fields loaded");
    const size_t n = (size_t)c->nx * c->ny * c->nz;
    RC(ensure_staging(c));
    CK(cudaDeviceSynchronize(), "wx_read_fields");
    RC(launch_unpack(c, c->fld[c->cur], T ? c->staging : nullptr, q ? c->staging + n : nullptr, 0));
    CK(cudaDeviceSynchronize(), "unpack");
    if (T) CK(cudaMemcpy(T, c->staging, n * sizeof(double), cudaMemcpyDeviceToHost), "download T");
    if (q) CK(cudaMemcpy(q, c->staging + n, n * sizeof(double), cudaMemcpyDeviceToHost), "download q");
    return WX_OK;
}

// FP32 state in and out (FP32-storage contexts): the step's inputs and
// results in their storage precision, half the bytes of the FP64 calls.
extern "C" int wx_load_state_f32(wx_ctx *c, const float *T, const float *q, int src_is_device) {
    if (!c) return WX_EINVAL;
    if (!T || !q) return fail(c, WX_EINVAL, "wx_load_state_f32: NULL array");
    if (c->t_bytes != 4) return fail(c, WX_EUNSUPPORTED, "wx_load_state_f32: the context stores FP64");
    if (!c->fields_loaded) return fail(c, WX_ESTATE, "wx_load_state_f32: load the winds with wx_load_fields first");
    const size_t n = (size_t)c->nx * c->ny * c->nz;
    const float *dT = T, *dq = q;
    if (!src_is_device) {
        RC(ensure_staging(c));  // 2n doubles: room for 2n floats
        float *sT = reinterpret_cast<float *>(c->staging), *sq = sT + n;
        CK(cudaMemcpy(sT, T, n * sizeof(float), cudaMemcpyHostToDevice), "upload T");
        CK(cudaMemcpy(sq, q, n * sizeof(float), cudaMemcpyHostToDevice), "upload q");
        dT = sT;
        dq = sq;
    }
    CK(cudaDeviceSynchronize(), "wx_load_state_f32");
    c->cur = 0;
    RC(launch_pack_f32(c, dT, dq, c->fld[0], 0));
    CK(cudaMemset(c->d_sums_count, 0, sizeof(long long)), "reset sums count");
    CK(cudaDeviceSynchronize(), "wx_load_state_f32");
    reset_surrogate_policy(c);
    ++c->generation;
    return WX_OK;
}

extern "C" int wx_read_state_f32(wx_ctx *c, float *T, float *q) {
    if (!c) return WX_EINVAL;
    if (c->t_bytes != 4) return fail(c, WX_EUNSUPPORTED, "wx_read_state_f32: the context stores FP64");
    if (!c->fields_loaded) return fail(c, WX_ESTATE, "wx_read_state_f32: no fields loaded");
    const size_t n = (size_t)c->nx * c->ny * c->nz;
    RC(ensure_staging(c));
    float *sT = reinterpret_cast<float *>(c->staging), *sq = sT + n;
    CK(cudaDeviceSynchronize(), "wx_read_state_f32");
    RC(launch_unpack_f32(c, c->fld[c->cur], T ? sT : nullptr, q ? sq : nullptr, 0));
    CK(cudaDeviceSynchronize(), "unpack");
    if (T) CK(cudaMemcpy(T, sT, n * sizeof(float), cudaMemcpyDeviceToHost), "download T");
    if (q) CK(cudaMemcpy(q, sq, n * sizeof(float), cudaMemcpyDeviceToHost), "download q");
    return WX_OK;
}

// The same on the caller's stream, without waiting: host arrays must be
// pinned (the copy engines read and write them while the host goes on), and
// stay untouched until the stream has passed the call.  Two contexts on two
// streams then overlap one's download with the other's upload.
static bool pinned_host(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

extern "C" int wx_load_state_f32_async(wx_ctx *c, const float *T, const float *q, void *stream) {
    if (!c) return WX_EINVAL;
    if (!T || !q) return fail(c, WX_EINVAL, "wx_load_state_f32_async: NULL array");
    if (c->t_bytes != 4) return fail(c, WX_EUNSUPPORTED, "wx_load_state_f32_async: the context stores FP64");
    if (!c->fields_loaded)
        return fail(c, WX_ESTATE, "wx_load_state_f32_async: load the winds with wx_load_fields first");
    if (!pinned_host(T) || !pinned_host(q))
        return fail(c, WX_EINVAL, "wx_load_state_f32_async: T and q must be pinned host memory");
    const size_t n = (size_t)c->nx * c->ny * c->nz;
    cudaStream_t s = (cudaStream_t)stream;
    RC(ensure_staging(c));  // 2n doubles: room for 2n floats
    float *sT = reinterpret_cast<float *>(c->staging), *sq = sT + n;
    CK(cudaMemcpyAsync(sT, T, n * sizeof(float), cudaMemcpyHostToDevice, s), "upload T");
    CK(cudaMemcpyAsync(sq, q, n * sizeof(float), cudaMemcpyHostToDevice, s), "upload q");
    c->cur = 0;
    RC(launch_pack_f32(c, sT, sq, c->fld[0], s));
    CK(cudaMemsetAsync(c->d_sums_count, 0, sizeof(long long), s), "reset sums count");
    reset_surrogate_policy(c);
    ++c->generation;
    c->last_stream = s;
    return WX_OK;
}

extern "C" int wx_read_state_f32_async(wx_ctx *c, float *T, float *q, void *stream) {
    if (!c) return WX_EINVAL;
    if (c->t_bytes != 4) return fail(c, WX_EUNSUPPORTED, "wx_read_state_f32_async: the context stores FP64");
    if (!c->fields_loaded) return fail(c, WX_ESTATE, "wx_read_state_f32_async: no fields loaded");
    if ((T && !pinned_host(T)) || (q && !pinned_host(q)))
        return fail(c, WX_EINVAL, "wx_read_state_f32_async: T and q must be pinned host memory");
    const size_t n = (size_t)c->nx * c->ny * c->nz;
    cudaStream_t s = (cudaStream_t)stream;
    RC(ensure_staging(c));
    float *sT = reinterpret_cast<float *>(c->staging), *sq = sT + n;
    RC(launch_unpack_f32(c, c->fld[c->cur], T ? sT : nullptr, q ? sq : nullptr, s));
    if (T) CK(cudaMemcpyAsync(T, sT, n * sizeof(float), cudaMemcpyDeviceToHost, s), "download T");
    if (q) CK(cudaMemcpyAsync(q, sq, n * sizeof(float), cudaMemcpyDeviceToHost, s), "download q");
    c->last_stream = s;
    return WX_OK;
}

// ------------------------------------------------------------ stepping
extern "C" int wx_step(wx_ctx *c, int n_steps, void *stream) {
    if (!c) return WX_EINVAL;
    if (n_steps < 0) return fail(c, WX_EINVAL, "wx_step: n_steps < 0");
    if (!c->params_set || !c->fields_loaded) return fail(c, WX_ESTATE, "wx_step: set params and load fields first");
    RC(check_cfl(c));
    cudaStream_t s = (cudaStream_t)stream;
    long launches = 0;
    if (c->flags & WX_SURROGATE) {
        if (!c->sur) return fail(c, WX_ESTATE, "wx_step: WX_SURROGATE without an attached network");
        for (int n = 0; n < n_steps; ++n) RC(launch_surrogate_policy_step(c, s, &launches));
    } else if (c->flags & WX_RK3) {
        for (int n = 0; n < n_steps; ++n) RC(launch_rk3_step(c, s, &launches));
    } else {
        for (int n = 0; n < n_steps; ++n) RC(launch_step(c, s, &launches));
    }
    c->last_launches = launches;
    c->last_stream = s;
    return WX_OK;
}

extern "C" int wx_sync(wx_ctx *c) {
    if (!c) return WX_EINVAL;
    CK(cudaStreamSynchronize(c->last_stream), "wx_sync");
    unsigned st = 0;
    CK(cudaMemcpy(&st, c->d_status, sizeof st, cudaMemcpyDeviceToHost), "read status");
    if (st) CK(cudaMemset(c->d_status, 0, sizeof(unsigned)), "clear status");
    if (st & ST_TIMEOUT) return fail(c, WX_ETIMEOUT, "a bounded device wait timed out");
    if (st & ST_BOUNDS) return fail(c, WX_ECUDA, "a kernel skipped an out-of-bounds access (bounds-checked build)");
    if (st & ST_NONFINITE) return fail(c, WX_ENONFINITE, "a step produced a non-finite value");
    if (st) return fail(c, WX_ECUDA, "device reported an invalid argument");
    return WX_OK;
}

extern "C" int wx_get_sums(wx_ctx *c, double *mass_q, double *energy_T, int max_steps, int *n_out) {
    if (!c) return WX_EINVAL;
    if (max_steps < 0) return fail(c, WX_EINVAL, "wx_get_sums: max_steps < 0");
    CK(cudaDeviceSynchronize(), "wx_get_sums");
    long long count = 0;
    CK(cudaMemcpy(&count, c->d_sums_count, sizeof count, cudaMemcpyDeviceToHost), "read sums count");
    const long avail = (long)std::min<long long>(count, c->sums_cap);
    const long n = std::min<long>(avail, max_steps);
    std::vector<double> ring(2 * (size_t)c->sums_cap);
    if (n > 0)
        CK(cudaMemcpy(ring.data(), c->sums_ring, ring.size() * sizeof(double), cudaMemcpyDeviceToHost),
           "download sums");
    for (long e = 0; e < n; ++e) {
        const long long step = count - n + e;
        const long slot = (long)(step % c->sums_cap);
        if (mass_q) mass_q[e] = ring[2 * slot];
        if (energy_T) energy_T[e] = ring[2 * slot + 1];
    }
    if (n_out) *n_out = (int)n;
    return WX_OK;
}

extern "C" int wx_physics_columns(wx_ctx *c, const void *Ts, const void *qs, const void *km, void *Tout,
                                  void *tend, long ncol, void *stream) {
    if (!c) return WX_EINVAL;
    if (ncol < 0) return fail(c, WX_EINVAL, "wx_physics_columns: ncol < 0");
    if (ncol > 0 && (!Ts || !qs || !Tout)) return fail(c, WX_EINVAL, "wx_physics_columns: NULL array");
    if (!c->params_set) return fail(c, WX_ESTATE, "wx_physics_columns: set params first");
    int rc = launch_columns(c, Ts, qs, km, Tout, tend, ncol, (cudaStream_t)stream);
    c->last_stream = (cudaStream_t)stream;
    return rc;
}


// ------------------------------------------------------------ self test
// A wait on an mbarrier that no thread will ever arrive on: the bounded
// wait every kernel of the library uses must give up after limit_ns, report
// it through the status word, and leave the context usable.
namespace wx {
__global__ void selftest_wait_kernel(uint64_t limit_ns, unsigned *status, unsigned long long *waited_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint64_t t0 = globaltimer_ns();
        const bool ok = mbar_wait_bounded(&bar, 0, limit_ns);
        *waited_ns = globaltimer_ns() - t0;
        if (!ok) atomicOr(status, ST_TIMEOUT);
    }
}
}  // namespace wx

extern "C" int wx_selftest_wait_timeout(unsigned long long limit_ns, unsigned long long *waited_ns) {
    if (!waited_ns || limit_ns == 0 || limit_ns > WX_SPIN_NS) return WX_EINVAL;
    unsigned *st = nullptr;
    unsigned long long *w = nullptr;
    if (cudaMalloc(&st, sizeof *st) != cudaSuccess || cudaMalloc(&w, sizeof *w) != cudaSuccess) {
        cudaFree(st);
        cudaGetLastError();
        return WX_ENOMEM;
    }
    cudaMemset(st, 0, sizeof *st);
    wx::selftest_wait_kernel<<<1, 32>>>(limit_ns, st, w);
    unsigned s = 0;
    const bool ok = cudaGetLastError() == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess &&
                    cudaMemcpy(&s, st, sizeof s, cudaMemcpyDeviceToHost) == cudaSuccess &&
                    cudaMemcpy(waited_ns, w, sizeof *w, cudaMemcpyDeviceToHost) == cudaSuccess;
    cudaFree(st);
    cudaFree(w);
    if (!ok) return WX_ECUDA;
    return (s & ST_TIMEOUT) ? WX_ETIMEOUT : WX_OK;
}
