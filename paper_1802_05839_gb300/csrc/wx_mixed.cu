// wx_mixed.cu -- the precision selection of WX_MIXED (and the kappa_mult
// side solve of WX_F32): which columns leave the step kernel's table path,
// their elimination factors, and the side solve that finishes them after
// each step.
//
// The step kernel runs every column on the kappa_mult = 1 table path and
// parks T* and dt H of the listed columns; the side solve then redoes the
// implicit vertical diffusion of those columns with their own matrix (in
// FP64 where the matrix is only weakly diagonally dominant) and overwrites
// their T (Sec. 2.1: the K recurrence stays sequential per column).
#include <vector>

#include "wx_internal.cuh"

namespace wx {

static int mixed_fail(wx_ctx *c, cudaError_t e, const char *what) {
    c->err = std::string(what) + ": " + cudaGetErrorString(e);
    return WX_ECUDA;
}

#define WX_CK(call, what)                                      \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return mixed_fail(c, e_, what); \
    } while (0)

// Dominance ratio of column (i, j): min_k |b_k| / (|a_k| + |c_k|) of its
// implicit vertical-diffusion matrix, in FP64.
__device__ double column_ratio(const double *lev, int nz, double dt, double km) {
    const double *dz = lev, *kl = lev + nz;
    double r = 1e300;
    for (int k = 0; k < nz; ++k) {
        double ak = 0, ck = 0;
        if (k > 0) ak = -dt * km * (0.5 * (kl[k - 1] + kl[k])) / (dz[k] * 0.5 * (dz[k - 1] + dz[k]));
        if (k < nz - 1) ck = -dt * km * (0.5 * (kl[k] + kl[k + 1])) / (dz[k] * 0.5 * (dz[k] + dz[k + 1]));
        const double off = fabs(ak) + fabs(ck);
        if (off > 0) r = fmin(r, fabs(1.0 - ak - ck) / off);
    }
    return r;
}

// One thread per column: 1 = FP64 solve (dominance ratio below the
// threshold), 2 = FP32 side solve (other kappa_mult != 1), 0 = neither.
__global__ void flag_class_kernel(const double *lev, const double *km, long ncol, int nz, double dt, double thr,
                                  unsigned char *cls) {
    const long col = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncol) return;
    const double s = km[col];
    cls[col] = column_ratio(lev, nz, dt, s) < thr ? 1 : (s != 1.0 ? 2 : 0);
}

// One thread per row: how many columns of each class row j holds.
__global__ void flag_count_kernel(const unsigned char *cls, int nx, int ny, int *count64, int *count32) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ny) return;
    int n64 = 0, n32 = 0;
    for (int i = 0; i < nx; ++i) {
        const unsigned char c = cls[(size_t)j * nx + i];
        n64 += c == 1;
        n32 += c == 2;
    }
    count64[j] = n64;
    count32[j] = n32;
}

// One thread per row: the row's listed columns in raster order from its
// offsets (FP64 columns first in the list, then the FP32 ones), -1 for the
// columns the step kernel finishes itself.
__global__ void flag_fill_kernel(const unsigned char *cls, const int *off64, const int *off32, int nx, int ny,
                                 int *list, int *idx) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ny) return;
    int f64 = off64[j], f32 = off32[j];
    for (int i = 0; i < nx; ++i) {
        const size_t col = (size_t)j * nx + i;
        const unsigned char c = cls[col];
        const int f = c == 1 ? f64++ : (c == 2 ? f32++ : -1);
        if (f >= 0) list[f] = (int)col;
        idx[col] = f;
    }
}

// One thread per listed column: the top-down elimination factors in FP64,
// m_k = b_k - c_k e_{k+1}, stored as (1/m_k, c_k/m_k) in fac[k][f], and
// e_k = a_k/m_k in fe[k][f] (level-major, so warps read them coalesced).
__global__ void flag_factor_kernel(const double *lev, const double *km, const int *list, long nflag, int nz,
                                   double dt, double2 *fac, float *fe) {
    const long f = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nflag) return;
    const double *dz = lev, *kl = lev + nz;
    const double s = km[list[f]];
    double e_up = 0.0;
    for (int k = nz - 1; k >= 0; --k) {
        double ak = 0, ck = 0;
        if (k > 0) ak = -dt * s * (0.5 * (kl[k - 1] + kl[k])) / (dz[k] * 0.5 * (dz[k - 1] + dz[k]));
        if (k < nz - 1) ck = -dt * s * (0.5 * (kl[k] + kl[k + 1])) / (dz[k] * 0.5 * (dz[k] + dz[k + 1]));
        const double inv = 1.0 / ((1.0 - ak - ck) - ck * e_up);
        const double e = ak * inv;
        fac[(size_t)k * nflag + f] = make_double2(inv, ck * inv);
        fe[(size_t)k * nflag + f] = (float)e;
        e_up = e;
    }
}

// Both sweeps go kSideChunk levels at a time: a chunk's loads (coalesced
// factors and parked values) are issued before its recurrence and stores,
// so that their latencies overlap.
constexpr int kSideChunk = 8;

// Elimination from the top, f_k = (T*_k - c_k f_{k+1}) / m_k with the
// column's precomputed (1/m_k, c_k/m_k): in FP64 (F = double) for weakly
// dominant columns, else in FP32.  r[k*st] holds T*_k; f_k (rounded to
// FP32) goes to fo[k*fst] (shared memory, or r itself).
template <typename F>
__device__ __forceinline__ void side_eliminate(const double2 *__restrict__ fac, const float *r, long nflag, long f,
                                               size_t st, int nz, float *fo, size_t fst) {
    F fu = F(0);
    for (int k0 = nz - 1; k0 >= 0; k0 -= kSideChunk) {
        double2 c2[kSideChunk];
        float ts[kSideChunk];
#pragma unroll
        for (int u = 0; u < kSideChunk; ++u) {
            const int k = k0 - u;
            c2[u] = k >= 0 ? fac[(size_t)k * nflag + f] : make_double2(0.0, 0.0);
            ts[u] = k >= 0 ? r[k * st] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kSideChunk; ++u) {
            const int k = k0 - u;
            if (k >= 0) {
                fu = fma(-(F)c2[u].y, fu, (F)c2[u].x * (F)ts[u]);  // (T*_k - c_k f_{k+1}) / m_k
                fo[k * fst] = (float)fu;
            }
        }
    }
}

// Back substitution from the bottom, x_k = f_k - e_k x_{k-1}, then T = x + dt*H
// into the column (i, j) of the new state `out` and its periodic ghost
// copies; with corr, the column's sum of T dz (dz as hi + lo floats, exact
// product error and TwoSum written as round-to-nearest intrinsics so that
// nothing is contracted) goes to corr[f].
__device__ __forceinline__ void side_back(const float *__restrict__ fe, const float *r, long nflag, long f,
                                          size_t st, const float *fi, size_t fst, int nz,
                                          const Q4<float> *__restrict__ dz2,
                                          float *__restrict__ out, int nx, int ny, int P, int R, int i, int j,
                                          double *__restrict__ corr, unsigned *status) {
    const size_t lev = (size_t)2 * R * P;
    const int ip = i + kGhostX;
    float *col0 = out + (size_t)(j + 1) * P;  // level 0 row of the column's T
    const long long out_n = (long long)lev * nz;
    auto put = [&](float *p, float v) {
        if (WX_IN(p - out, out_n, status)) *p = v;
    };
    float x = 0.f;
    float sE = 0.f, cE = 0.f;  // compensated sum of T dz
    for (int k0 = 0; k0 < nz; k0 += kSideChunk) {
        float fk[kSideChunk], ek[kSideChunk], hk[kSideChunk];
#pragma unroll
        for (int u = 0; u < kSideChunk; ++u) {
            const int k = k0 + u;
            const bool in = k < nz;
            ek[u] = in ? fe[(size_t)k * nflag + f] : 0.f;
            fk[u] = in ? fi[k * fst] : 0.f;
            hk[u] = in ? r[k * st + nflag] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kSideChunk; ++u) {
            const int k = k0 + u;
            if (k >= nz) break;
            x = fmaf(-ek[u], x, fk[u]);
            const float tn = x + hk[u];
            float *row = col0 + k * lev;
            if (corr) {
                const float dzh = dz2[k].z, dzl = dz2[k].w;
                const float p = __fmul_rn(tn, dzh);
                const float pe = __fmaf_rn(tn, dzl, __fmaf_rn(tn, dzh, -p));
                const float s1 = __fadd_rn(sE, p), bp = __fsub_rn(s1, sE);
                const float e = __fadd_rn(__fsub_rn(sE, __fsub_rn(s1, bp)), __fsub_rn(p, bp));
                cE = __fadd_rn(cE, __fadd_rn(e, pe));
                sE = s1;
            }
            put(row + ip, tn);
            if (i == 0) put(row + kGhostX + nx, tn);
            if (i == nx - 1) put(row + kGhostX - 1, tn);
            if (j == 0) put(out + k * lev + (size_t)(ny + 1) * P + ip, tn);
            if (j == ny - 1) put(out + k * lev + ip, tn);
        }
    }
    if (corr) corr[f] = (double)sE + (double)cE;
}

// The whole side solve of listed column f (column index col = j*nx + i);
// fb[k*fst] holds f_k between the sweeps.
__device__ __forceinline__ void side_column(const int *__restrict__ list, long nflag, long n64,
                                            const double2 *__restrict__ fac, const float *__restrict__ fe,
                                            const float *__restrict__ side, const Q4<float> *__restrict__ dz2,
                                            float *__restrict__ out, double *__restrict__ corr, int nx, int ny,
                                            int nz, int P, int R, long f, float *fb, size_t fst, unsigned *status) {
    const int col = list[f], i = col % nx, j = col / nx;
    if (!WX_IN(col, (long long)nx * ny, status)) return;
    const float *r = side + f;  // r[2k*nflag]: T*_k; r[(2k+1)*nflag]: dt*H_k
    const size_t st = 2 * (size_t)nflag;
    if (f < n64)
        side_eliminate<double>(fac, r, nflag, f, st, nz, fb, fst);  // weakly dominant: FP64
    else
        side_eliminate<float>(fac, r, nflag, f, st, nz, fb, fst);   // other kappa_mult != 1 columns
    side_back(fe, r, nflag, f, st, fb, fst, nz, dz2, out, nx, ny, P, R, i, j, corr, status);
}

// One thread per listed column (warps of listed work only): the side solve
// above.  The column's T (and its ghost copies) in the new state is
// overwritten; with sums, the column's own FP64 sum of T dz is recorded for
// the finalize kernel (the step kernel leaves listed columns out of its T
// sums).  With nz <= kFixSmemNz the f_k stay in shared memory between the
// sweeps ([k][thread]); otherwise they overwrite the parked T* in place.
constexpr int kFixThreads = 128, kFixSmemNz = 64;
template <bool SM>
__global__ void __launch_bounds__(kFixThreads, 6) mixed_fixup_kernel(const int *__restrict__ list, long nflag, long n64,
                                                          const double2 *__restrict__ fac,
                                                          const float *__restrict__ fe, float *__restrict__ side,
                                                          const Q4<float> *__restrict__ dz2, float *__restrict__ out,
                                                          double *__restrict__ corr, int nx, int ny, int nz, int P,
                                                          int R, unsigned *__restrict__ status) {
    extern __shared__ float fsh[];
    const long f = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nflag) return;
    if (SM)
        side_column(list, nflag, n64, fac, fe, side, dz2, out, corr, nx, ny, nz, P, R, f, fsh + threadIdx.x,
                    (size_t)kFixThreads, status);
    else
        side_column(list, nflag, n64, fac, fe, side, dz2, out, corr, nx, ny, nz, P, R, f, side + f,
                    2 * (size_t)nflag, status);
}

int launch_mixed_fixup(wx_ctx *c, int dst, bool sums, cudaStream_t s) {
    const int nt = kFixThreads;
    const bool sm = c->nz <= kFixSmemNz;
    auto kern = sm ? mixed_fixup_kernel<true> : mixed_fixup_kernel<false>;
    if (sm && !c->fixup_carveout) {  // six blocks' f_k in shared memory per SM (once per context)
        WX_CK(cudaFuncSetAttribute(mixed_fixup_kernel<true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                   cudaSharedmemCarveoutMaxShared),
              "fixup carveout");
        c->fixup_carveout = true;
    }
    kern<<<(unsigned)((c->n_list + nt - 1) / nt), nt, sm ? (size_t)nt * c->nz * sizeof(float) : 0, s>>>(
        c->flag_list, c->n_list, c->n_flag, (const double2 *)c->flag_fac, c->flag_e, c->flag_side,
        (const Q4<float> *)c->tab + REC_F * c->nz, (float *)c->fld[dst], sums ? c->flag_corr : nullptr, c->nx,
        c->ny, c->nz, c->P, c->R, c->d_status);
    WX_CK(cudaGetLastError(), "mixed fixup kernel");
    return WX_OK;
}

// WX_MIXED set-up: flag the columns whose dominance ratio is below the
// threshold (deterministic raster order) and precompute their FP64 factors.
// km64 is the FP64 kappa_mult on the device.
int setup_mixed(wx_ctx *c, const double *km64) {
    for (void **p : {(void **)&c->flag_list, (void **)&c->flag_idx, (void **)&c->flag_fac, (void **)&c->flag_e,
                     (void **)&c->flag_side, (void **)&c->flag_corr})
        if (*p) {
            cudaFree(*p);
            *p = nullptr;
        }
    c->n_flag = c->n_list = 0;
    if ((c->dtype != WX_MIXED && c->dtype != WX_F32) || !km64) return WX_OK;
    // WX_F32 lists the kappa_mult != 1 columns but solves none of them in FP64
    const double thr = c->dtype == WX_MIXED ? c->dd_threshold : 0.0;
    const int ny = c->ny, nx = c->nx, nz = c->nz;
    const size_t ncol = (size_t)nx * ny;
    int *d_cnt = nullptr;  // [4][ny]: count64, count32, off64, off32; then the classes
    WX_CK(cudaMalloc(&d_cnt, 4 * (size_t)ny * sizeof(int) + ncol), "alloc flag counts");
    struct Scratch {
        void *p;
        ~Scratch() { cudaFree(p); }
    } scratch{d_cnt};  // freed on every return below
    unsigned char *cls = reinterpret_cast<unsigned char *>(d_cnt + 4 * (size_t)ny);
    flag_class_kernel<<<(unsigned)((ncol + 255) / 256), 256>>>(c->d_lev, km64, (long)ncol, nz, c->dt, thr, cls);
    flag_count_kernel<<<(ny + 127) / 128, 128>>>(cls, nx, ny, d_cnt, d_cnt + ny);
    std::vector<int> cnt(2 * (size_t)ny), off(2 * (size_t)ny);
    cudaError_t e = cudaMemcpy(cnt.data(), d_cnt, 2 * ny * sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return mixed_fail(c, e, "flag counts");
    long n64 = 0, n32 = 0;
    for (int j = 0; j < ny; ++j) n64 += cnt[j];
    long a64 = 0, a32 = n64;
    for (int j = 0; j < ny; ++j) {
        off[j] = (int)a64;
        a64 += cnt[j];
        off[ny + j] = (int)a32;
        a32 += cnt[ny + j];
        n32 += cnt[ny + j];
    }
    const long n = n64 + n32;
    WX_CK(cudaMalloc(&c->flag_idx, (size_t)nx * ny * sizeof(int)), "alloc flag index");
    if (n > 0) {
        WX_CK(cudaMalloc(&c->flag_list, n * sizeof(int)), "alloc flag list");
        WX_CK(cudaMalloc(&c->flag_fac, (size_t)n * nz * 2 * sizeof(double)), "alloc flag factors");
        WX_CK(cudaMalloc(&c->flag_e, (size_t)n * nz * sizeof(float)), "alloc flag e");
        WX_CK(cudaMalloc(&c->flag_side, (size_t)n * 2 * nz * sizeof(float)), "alloc flag side buffer");
        WX_CK(cudaMalloc(&c->flag_corr, (size_t)n * sizeof(double)), "alloc flag corrections");
    }
    WX_CK(cudaMemcpy(d_cnt + 2 * ny, off.data(), 2 * ny * sizeof(int), cudaMemcpyHostToDevice), "flag offsets");
    flag_fill_kernel<<<(ny + 127) / 128, 128>>>(cls, d_cnt + 2 * ny, d_cnt + 3 * ny, nx, ny, c->flag_list,
                                                c->flag_idx);
    if (n > 0)
        flag_factor_kernel<<<(unsigned)((n + 127) / 128), 128>>>(c->d_lev, km64, c->flag_list, n, nz, c->dt,
                                                                  (double2 *)c->flag_fac, c->flag_e);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return mixed_fail(c, e, "mixed-precision set-up");
    c->n_flag = n64;  // only now: a failed set-up leaves no listed columns
    c->n_list = n;
    return WX_OK;
}

}  // namespace wx
