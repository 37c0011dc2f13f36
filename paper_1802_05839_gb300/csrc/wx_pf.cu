// wx_pf.cu -- the paper's reduced weather application on the GPU.
//
// State: E[k][j][i] over i in [0, nx+2), j in [0, ny+2), k in [0, nz): the
// listings' arrays with their ghost ring, which is state of its own (it
// evolves by a two-neighbour rule, not by copying).  One step is the time
// loop of the appendix listings: the physics (uniform radiation on every
// level, Newtonian heat wells at the bottom and top levels) in place on
// every column, then diffusion into the other buffer, then the swap.
//
// The physics is pointwise and affine per level,
//   P_k(x) = a_k x + b_k,   a_k = 1, b_k = r for 0 < k < nz-1,
//   a_k = 1 - tau, b_k = (1 - tau) r + tau T_well at k = 0 (T_surf) and
//   k = nz-1 (T_pbl),
// so one kernel applies it to every value it reads: a sum of n neighbours
// at one level is P applied to their raw sum, a_k S + n b_k.  Each thread
// owns kPfChunk levels of one (i, j) column and walks them bottom to top,
// keeping the physics result of levels k-1, k, k+1 of its own column in
// registers; the four horizontal neighbours come from L1/L2 (a warp reads
// 32 consecutive i).  Splitting columns into chunks (grid z) keeps enough
// independent loads in flight: a whole column per thread leaves too few
// threads, each waiting on one level at a time.
//
// Two storage orders are kept for the paper's storage-order experiment
// (Sec. 2.4.3, Sec. 5.1.1): IJK (i fastest, the default: a warp's loads of
// one level are contiguous) and KIJ (k fastest, the CPU order: a warp's
// loads are nz cells apart).  The kernel is written once in terms of the
// strides (si, sj, sk) of the chosen order; the block shape is a launch
// parameter (the paper's block-size experiment, Sec. 5.1.4).
#include <algorithm>
#include <cmath>
#include <new>
#include <string>

#include "../../include/wx.h"

struct wx_pf {
    int nx = 0, ny = 0, nz = 0, dtype = 0;
    int W = 0, H = 0, P = 0;      // row width nx+2, rows ny+2, row pitch (cells, IJK)
    int layout = 0;               // WX_PF_IJK or WX_PF_KIJ
    int bx = 32, by = 8;          // thread-block shape
    size_t cells = 0, bytes = 0;  // per buffer (pitched)
    int tb = 0;                   // bytes per value
    void *buf[2] = {nullptr, nullptr};
    int cur = 0;
    double *staging = nullptr;    // FP64 [nz][H][W] for load / read
    unsigned *status = nullptr;
    double d = 0.1, r = 0.1, tau = 0.01, Ts = 330.0, Tp = 200.0;
    bool loaded = false;
    cudaStream_t last = nullptr;
    long launches = 0;
    std::string err;
};

namespace wxpf {

constexpr int kPfChunk = 8;  // levels per thread

template <typename T> struct PfArgs {
    const T *E;
    T *En;
    int nx, ny, nz, W, H;
    long si, sj, sk;                 // strides of i, j, k in the storage order
    T d, c6, c5, c2;                 // d, 1-6d, 1-5d, 1-2d
    T a_mid, b_mid, a_bot, b_bot, a_top, b_top;
    unsigned *status;
};

template <typename T>
__global__ void __launch_bounds__(512) pf_step_kernel(const PfArgs<T> g) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k0 = blockIdx.z * kPfChunk, k1 = min(k0 + kPfChunk, g.nz);
    if (i >= g.W || j >= g.H) return;
    const long plane = g.sk;
    // the two buffers never overlap: without __restrict__ every load would
    // wait for the previous level's store
    const T *__restrict__ E = g.E;
    T *__restrict__ En = g.En;
    const T *__restrict__ col = E + j * g.sj + i * g.si;
    T *__restrict__ out = En + j * g.sj + i * g.si;
    const bool ghost_col = (i == 0 || i == g.nx + 1);
    const bool ghost_row = !ghost_col && (j == 0 || j == g.ny + 1);
    auto aff_a = [&](int k) { return k == 0 ? g.a_bot : (k == g.nz - 1 ? g.a_top : g.a_mid); };
    auto aff_b = [&](int k) { return k == 0 ? g.b_bot : (k == g.nz - 1 ? g.b_top : g.b_mid); };
    bool finite = true;
    if (ghost_col || ghost_row) {
        // two neighbours on the same level: the row's (or column's) other end
        // and the adjacent interior cell
        const T *__restrict__ na;
        const T *__restrict__ nb;
        if (ghost_col) {
            na = E + j * g.sj + (i == 0 ? 1 : g.nx) * g.si;
            nb = E + j * g.sj + (i == 0 ? g.nx + 1 : 0) * g.si;
        } else {
            na = E + (j == 0 ? 1 : g.ny) * g.sj + i * g.si;
            nb = E + (j == 0 ? g.ny + 1 : 0) * g.sj + i * g.si;
        }
#pragma unroll 4
        for (int k = k0; k < k1; ++k) {
            const long o = k * plane;
            const T a = aff_a(k), b = aff_b(k);
            const T pc = a * col[o] + b;
            const T ps = a * (na[o] + nb[o]) + 2 * b;
            const T v = g.c2 * pc + g.d * ps;
            finite = finite && isfinite(v);
            out[o] = v;
        }
    } else {
        // interior column: 7-point rule, one-sided at the bottom and top
        T pm = k0 > 0 ? aff_a(k0 - 1) * col[(k0 - 1) * plane] + aff_b(k0 - 1) : T(0);
        T pc = aff_a(k0) * col[k0 * plane] + aff_b(k0);
#pragma unroll 4
        for (int k = k0; k < k1; ++k) {
            const long o = k * plane;
            const T a = aff_a(k), b = aff_b(k);
            const T pu = k + 1 < g.nz ? aff_a(k + 1) * col[o + plane] + aff_b(k + 1) : T(0);
            const T hs = (col[o - g.si] + col[o + g.si]) + (col[o - g.sj] + col[o + g.sj]);
            const T ph = a * hs + 4 * b;
            T v;
            if (k == 0)
                v = g.c5 * pc + g.d * (ph + pu);
            else if (k == g.nz - 1)
                v = g.c5 * pc + g.d * (ph + pm);
            else
                v = g.c6 * pc + g.d * (ph + (pm + pu));
            finite = finite && isfinite(v);
            out[o] = v;
            pm = pc;
            pc = pu;
        }
    }
    if (!finite) atomicOr(g.status, 1u);
}

// element e of the [nz][H][W] exchange order -> its offset in the storage order
__device__ __forceinline__ long pf_offset(size_t e, int W, int H, long si, long sj, long sk) {
    const long i = (long)(e % W), j = (long)((e / W) % H), k = (long)(e / ((size_t)W * H));
    return i * si + j * sj + k * sk;
}

template <typename T> __global__ void pf_pack_kernel(const double *__restrict__ src, T *__restrict__ dst, int W,
                                                     int H, int nz, long si, long sj, long sk) {
    const size_t n = (size_t)W * H * nz;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        dst[pf_offset(e, W, H, si, sj, sk)] = (T)src[e];
}

template <typename T> __global__ void pf_unpack_kernel(const T *__restrict__ src, double *__restrict__ dst, int W,
                                                       int H, int nz, long si, long sj, long sk) {
    const size_t n = (size_t)W * H * nz;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        dst[e] = (double)src[pf_offset(e, W, H, si, sj, sk)];
}

// strides of the storage order: IJK [k][j][P], KIJ [j][i][nz]
static void strides(const wx_pf *p, long *si, long *sj, long *sk) {
    if (p->layout == WX_PF_KIJ) {
        *sk = 1;
        *si = p->nz;
        *sj = (long)p->W * p->nz;
    } else {
        *si = 1;
        *sj = p->P;
        *sk = (long)p->H * p->P;
    }
}

template <typename T> static PfArgs<T> args(const wx_pf *p) {
    PfArgs<T> g;
    g.E = (const T *)p->buf[p->cur];
    g.En = (T *)p->buf[1 - p->cur];
    g.nx = p->nx;
    g.ny = p->ny;
    g.nz = p->nz;
    g.W = p->W;
    g.H = p->H;
    strides(p, &g.si, &g.sj, &g.sk);
    g.d = (T)p->d;
    g.c6 = (T)(1.0 - 6 * p->d);
    g.c5 = (T)(1.0 - 5 * p->d);
    g.c2 = (T)(1.0 - 2 * p->d);
    g.a_mid = (T)1.0;
    g.b_mid = (T)p->r;
    g.a_bot = (T)(1.0 - p->tau);
    g.b_bot = (T)((1.0 - p->tau) * p->r + p->tau * p->Ts);
    g.a_top = (T)(1.0 - p->tau);
    g.b_top = (T)((1.0 - p->tau) * p->r + p->tau * p->Tp);
    g.status = p->status;
    return g;
}

static int grid1(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 65535 * 8); }

}  // namespace wxpf

using namespace wxpf;

static int pfail(wx_pf *p, int code, const std::string &m) {
    if (p) p->err = m;
    return code;
}

#define PCK(call, what)                                                                                \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return pfail(p, WX_ECUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
    } while (0)

extern "C" void wx_pf_destroy(wx_pf *p) {
    if (!p) return;
    for (void *q : {p->buf[0], p->buf[1], (void *)p->staging, (void *)p->status})
        if (q) cudaFree(q);
    delete p;
}

extern "C" int wx_pf_create(int nx, int ny, int nz, int dtype, wx_pf **out) {
    if (!out) return WX_EINVAL;
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 2 || (dtype != WX_F32 && dtype != WX_F64)) return WX_EINVAL;
    if ((size_t)(nx + 2) * (ny + 2) * nz > (size_t)1 << 34) return WX_EUNSUPPORTED;
    wx_pf *p = new (std::nothrow) wx_pf();
    if (!p) return WX_ENOMEM;
    p->nx = nx;
    p->ny = ny;
    p->nz = nz;
    p->dtype = dtype;
    p->tb = dtype == WX_F64 ? 8 : 4;
    p->W = nx + 2;
    p->H = ny + 2;
    p->P = (p->W + 31) / 32 * 32;
    p->cells = std::max((size_t)p->P * p->H * nz, (size_t)p->W * p->H * nz);
    p->bytes = p->cells * p->tb;
    bool ok = cudaMalloc(&p->buf[0], p->bytes) == cudaSuccess && cudaMalloc(&p->buf[1], p->bytes) == cudaSuccess &&
              cudaMalloc((void **)&p->staging, (size_t)p->W * p->H * nz * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void **)&p->status, sizeof(unsigned)) == cudaSuccess &&
              cudaMemset(p->status, 0, sizeof(unsigned)) == cudaSuccess &&
              cudaMemset(p->buf[0], 0, p->bytes) == cudaSuccess && cudaMemset(p->buf[1], 0, p->bytes) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        wx_pf_destroy(p);
        return WX_ENOMEM;
    }
    *out = p;
    return WX_OK;
}

extern "C" int wx_pf_set_params(wx_pf *p, double d, double radiation, double transfer, double T_surf,
                                double T_pbl) {
    if (!p) return WX_EINVAL;
    if (!std::isfinite(d) || !std::isfinite(radiation) || !std::isfinite(transfer) || !std::isfinite(T_surf) ||
        !std::isfinite(T_pbl))
        return pfail(p, WX_EINVAL, "wx_pf_set_params: non-finite parameter");
    // the explicit update is a convex combination only for these ranges
    if (d < 0 || d > 1.0 / 6.0 || transfer < 0 || transfer > 1)
        return pfail(p, WX_ECFL, "wx_pf_set_params: need 0 <= d <= 1/6 and 0 <= transfer <= 1");
    p->d = d;
    p->r = radiation;
    p->tau = transfer;
    p->Ts = T_surf;
    p->Tp = T_pbl;
    return WX_OK;
}

extern "C" int wx_pf_load(wx_pf *p, const double *E, int src_is_device) {
    if (!p || !E) return pfail(p, WX_EINVAL, "wx_pf_load: NULL");
    const size_t n = (size_t)p->W * p->H * p->nz;
    PCK(cudaMemcpy(p->staging, E, n * sizeof(double), src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice),
        "wx_pf_load copy");
    long si, sj, sk;
    strides(p, &si, &sj, &sk);
    if (p->dtype == WX_F64)
        pf_pack_kernel<double><<<grid1(n), 256>>>(p->staging, (double *)p->buf[0], p->W, p->H, p->nz, si, sj, sk);
    else
        pf_pack_kernel<float><<<grid1(n), 256>>>(p->staging, (float *)p->buf[0], p->W, p->H, p->nz, si, sj, sk);
    PCK(cudaGetLastError(), "wx_pf_load pack");
    PCK(cudaDeviceSynchronize(), "wx_pf_load");
    p->cur = 0;
    p->loaded = true;
    return WX_OK;
}

extern "C" int wx_pf_read(wx_pf *p, double *E) {
    if (!p || !E) return pfail(p, WX_EINVAL, "wx_pf_read: NULL");
    if (!p->loaded) return pfail(p, WX_ESTATE, "wx_pf_read: nothing loaded");
    PCK(cudaDeviceSynchronize(), "wx_pf_read");
    const size_t n = (size_t)p->W * p->H * p->nz;
    long si, sj, sk;
    strides(p, &si, &sj, &sk);
    if (p->dtype == WX_F64)
        pf_unpack_kernel<double><<<grid1(n), 256>>>((const double *)p->buf[p->cur], p->staging, p->W, p->H, p->nz, si,
                                                    sj, sk);
    else
        pf_unpack_kernel<float><<<grid1(n), 256>>>((const float *)p->buf[p->cur], p->staging, p->W, p->H, p->nz, si,
                                                   sj, sk);
    PCK(cudaGetLastError(), "wx_pf_read unpack");
    PCK(cudaMemcpy(E, p->staging, n * sizeof(double), cudaMemcpyDeviceToHost), "wx_pf_read copy");
    return WX_OK;
}

extern "C" int wx_pf_step(wx_pf *p, int n_steps, void *stream) {
    if (!p) return WX_EINVAL;
    if (n_steps < 0) return pfail(p, WX_EINVAL, "wx_pf_step: n_steps < 0");
    if (!p->loaded) return pfail(p, WX_ESTATE, "wx_pf_step: load a state first");
    cudaStream_t s = (cudaStream_t)stream;
    const dim3 block(p->bx, p->by),
        grid((p->W + p->bx - 1) / p->bx, (p->H + p->by - 1) / p->by, (p->nz + kPfChunk - 1) / kPfChunk);
    for (int n = 0; n < n_steps; ++n) {
        if (p->dtype == WX_F64)
            pf_step_kernel<double><<<grid, block, 0, s>>>(args<double>(p));
        else
            pf_step_kernel<float><<<grid, block, 0, s>>>(args<float>(p));
        PCK(cudaGetLastError(), "wx_pf_step");
        p->cur = 1 - p->cur;
    }
    p->last = s;
    p->launches = n_steps;
    return WX_OK;
}

extern "C" int wx_pf_sync(wx_pf *p) {
    if (!p) return WX_EINVAL;
    PCK(cudaStreamSynchronize(p->last), "wx_pf_sync");
    unsigned st = 0;
    PCK(cudaMemcpy(&st, p->status, sizeof st, cudaMemcpyDeviceToHost), "wx_pf_sync status");
    if (st) {
        cudaMemset(p->status, 0, sizeof st);
        return pfail(p, WX_ENONFINITE, "a step produced a non-finite value");
    }
    return WX_OK;
}

// Storage order and block shape; a loaded state is carried over.
extern "C" int wx_pf_set_launch(wx_pf *p, int layout, int block_x, int block_y) {
    if (!p) return WX_EINVAL;
    if ((layout != WX_PF_IJK && layout != WX_PF_KIJ) || block_x < 1 || block_y < 1 || block_x * block_y > 512 ||
        block_x * block_y % 32)
        return pfail(p, WX_EINVAL, "wx_pf_set_launch: layout IJK/KIJ, block of 32..512 threads (multiple of 32)");
    if (p->loaded && layout != p->layout) {
        PCK(cudaDeviceSynchronize(), "wx_pf_set_launch");
        const size_t n = (size_t)p->W * p->H * p->nz;
        long si, sj, sk;
        strides(p, &si, &sj, &sk);
        if (p->dtype == WX_F64)
            pf_unpack_kernel<double><<<grid1(n), 256>>>((const double *)p->buf[p->cur], p->staging, p->W, p->H,
                                                        p->nz, si, sj, sk);
        else
            pf_unpack_kernel<float><<<grid1(n), 256>>>((const float *)p->buf[p->cur], p->staging, p->W, p->H, p->nz,
                                                       si, sj, sk);
        p->layout = layout;
        strides(p, &si, &sj, &sk);
        if (p->dtype == WX_F64)
            pf_pack_kernel<double><<<grid1(n), 256>>>(p->staging, (double *)p->buf[p->cur], p->W, p->H, p->nz, si,
                                                      sj, sk);
        else
            pf_pack_kernel<float><<<grid1(n), 256>>>(p->staging, (float *)p->buf[p->cur], p->W, p->H, p->nz, si,
                                                     sj, sk);
        PCK(cudaGetLastError(), "wx_pf_set_launch re-layout");
        PCK(cudaDeviceSynchronize(), "wx_pf_set_launch");
    }
    p->layout = layout;
    p->bx = block_x;
    p->by = block_y;
    return WX_OK;
}

extern "C" long wx_pf_last_launches(const wx_pf *p) { return p ? p->launches : 0; }

extern "C" const char *wx_pf_last_error(const wx_pf *p) { return p ? p->err.c_str() : "NULL handle"; }
