// wx_io.cu -- moving the state between the caller's [nz][ny][nx] arrays and
// the resident padded planar fields (with the periodic ghost ring).
//
// Host arrays travel through a device staging buffer by the copy engines
// (about 200 GB/s each way over the host link, measured; kernels reading or
// writing pinned host memory in place were slower: 168 GB/s in, 120 GB/s
// out).  The kernels run one padded row per block iteration (no
// per-element index division), four independent loads per thread.
#include "wx_internal.cuh"

namespace wx {

constexpr int kIoThreads = 256;
constexpr int kIoUnroll = 4;

// dst row r = (2k + f) R + jp holds field f (T, q) of level k at padded row
// jp; its interior starts kGhostX cells in, with one periodic ghost column
// on either side and zeros elsewhere.  Rows jp = 0 and ny+1 are the
// periodic copies of rows ny-1 and 0.
template <typename T, typename S>
__global__ void __launch_bounds__(kIoThreads) pack_rows_kernel(const S *__restrict__ Tsrc,
                                                               const S *__restrict__ qsrc, T *__restrict__ dst,
                                                               int nx, int ny, int nz, int P, int R) {
    const long rows = 2L * nz * R;
    for (long r = blockIdx.x; r < rows; r += gridDim.x) {
        const int jp = (int)(r % R);
        const int f = (int)((r / R) & 1);
        const int k = (int)(r / (2L * R));
        const int j = jp == 0 ? ny - 1 : (jp == ny + 1 ? 0 : jp - 1);
        const S *src = (f == 0 ? Tsrc : qsrc) + ((size_t)k * ny + j) * nx;
        T *out = dst + (size_t)r * P;
        for (int ip0 = threadIdx.x; ip0 < P; ip0 += kIoUnroll * kIoThreads) {
            T v[kIoUnroll];
#pragma unroll
            for (int u = 0; u < kIoUnroll; ++u) {
                const int i = ip0 + u * kIoThreads - kGhostX;
                v[u] = (i >= -1 && i <= nx) ? (T)src[i < 0 ? nx - 1 : (i == nx ? 0 : i)] : (T)0;
            }
#pragma unroll
            for (int u = 0; u < kIoUnroll; ++u)
                if (ip0 + u * kIoThreads < P) out[ip0 + u * kIoThreads] = v[u];
        }
    }
}

// Interior of the padded fields -> [nz][ny][nx] (T, q); either output may be null.
template <typename T, typename D>
__global__ void __launch_bounds__(kIoThreads) unpack_rows_kernel(const T *__restrict__ src, D *__restrict__ Tdst,
                                                                 D *__restrict__ qdst, int nx, int ny, int nz,
                                                                 int P, int R) {
    const long rows = (long)nz * ny;
    for (long r = blockIdx.x; r < rows; r += gridDim.x) {
        const int j = (int)(r % ny);
        const int k = (int)(r / ny);
        const T *sT = src + ((size_t)(2 * k) * R + j + 1) * P + kGhostX;
        const T *sq = sT + (size_t)R * P;
        const size_t o = (size_t)r * nx;
        for (int i0 = threadIdx.x; i0 < nx; i0 += kIoUnroll * kIoThreads) {
#pragma unroll
            for (int u = 0; u < kIoUnroll; ++u) {
                const int i = i0 + u * kIoThreads;
                if (i < nx) {
                    if (Tdst) Tdst[o + i] = (D)sT[i];
                    if (qdst) qdst[o + i] = (D)sq[i];
                }
            }
        }
    }
}

template <typename T> __global__ void convert_kernel(const double *__restrict__ s, T *__restrict__ d, size_t n) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        d[e] = (T)s[e];
}

static int io_fail(wx_ctx *c, cudaError_t e, const char *what) {
    c->err = std::string(what) + ": " + cudaGetErrorString(e);
    return WX_ECUDA;
}

#define IO_CK(call, what)                                   \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return io_fail(c, e_, what); \
    } while (0)

// Blocks for `rows` rows: up to 8 resident 256-thread blocks on every SM.
static int io_blocks(long rows) {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long cap = 8L * sms;
    return (int)(rows < 1 ? 1 : (rows < cap ? rows : cap));
}

int launch_pack(wx_ctx *c, const double *T, const double *q, void *dst, cudaStream_t s) {
    const int g = io_blocks(2L * c->nz * c->R);
    if (c->t_bytes == 4)
        pack_rows_kernel<float, double>
            <<<g, kIoThreads, 0, s>>>(T, q, (float *)dst, c->nx, c->ny, c->nz, c->P, c->R);
    else
        pack_rows_kernel<double, double>
            <<<g, kIoThreads, 0, s>>>(T, q, (double *)dst, c->nx, c->ny, c->nz, c->P, c->R);
    IO_CK(cudaGetLastError(), "pack kernel");
    return WX_OK;
}

int launch_unpack(wx_ctx *c, const void *src, double *T, double *q, cudaStream_t s) {
    const int g = io_blocks((long)c->nz * c->ny);
    if (c->t_bytes == 4)
        unpack_rows_kernel<float, double>
            <<<g, kIoThreads, 0, s>>>((const float *)src, T, q, c->nx, c->ny, c->nz, c->P, c->R);
    else
        unpack_rows_kernel<double, double>
            <<<g, kIoThreads, 0, s>>>((const double *)src, T, q, c->nx, c->ny, c->nz, c->P, c->R);
    IO_CK(cudaGetLastError(), "unpack kernel");
    return WX_OK;
}

// FP32 state of an FP32-storage context (no conversion on the way).
int launch_pack_f32(wx_ctx *c, const float *T, const float *q, void *dst, cudaStream_t s) {
    pack_rows_kernel<float, float><<<io_blocks(2L * c->nz * c->R), kIoThreads, 0, s>>>(
        T, q, (float *)dst, c->nx, c->ny, c->nz, c->P, c->R);
    IO_CK(cudaGetLastError(), "pack kernel");
    return WX_OK;
}

int launch_unpack_f32(wx_ctx *c, const void *src, float *T, float *q, cudaStream_t s) {
    unpack_rows_kernel<float, float><<<io_blocks((long)c->nz * c->ny), kIoThreads, 0, s>>>(
        (const float *)src, T, q, c->nx, c->ny, c->nz, c->P, c->R);
    IO_CK(cudaGetLastError(), "unpack kernel");
    return WX_OK;
}

int launch_convert(wx_ctx *c, const double *src, void *dst, size_t n, cudaStream_t s) {
    const size_t b = (n + kIoThreads - 1) / kIoThreads;
    const int g = (int)(b < 1 ? 1 : (b > 65535 ? 65535 : b));
    if (c->t_bytes == 4)
        convert_kernel<float><<<g, kIoThreads, 0, s>>>(src, (float *)dst, n);
    else
        convert_kernel<double><<<g, kIoThreads, 0, s>>>(src, (double *)dst, n);
    IO_CK(cudaGetLastError(), "convert kernel");
    return WX_OK;
}

// The state as FP32 columns dst[col][k], col = j nx + i: a block stages the
// planes of 32 consecutive columns (each level's read coalesced along x),
// then writes each column's nz values contiguously.
template <typename T>
__global__ void __launch_bounds__(kIoThreads) columns_out_kernel(const T *__restrict__ src, float *__restrict__ Tdst,
                                                                 float *__restrict__ qdst, int nx, int nz, int P,
                                                                 int R, long ncol) {
    extern __shared__ float cs[];  // [nz][33]
    const long c0 = (long)blockIdx.x * 32;
    for (int f = 0; f < 2; ++f) {
        float *dst = f ? qdst : Tdst;
        if (!dst) continue;
        __syncthreads();
        for (int e = threadIdx.x; e < nz * 32; e += blockDim.x) {
            const int k = e / 32, u = e % 32;
            const long c = c0 + u;
            float v = 0.f;
            if (c < ncol) {
                const int j = (int)(c / nx), i = (int)(c - (long)j * nx);
                v = (float)src[((size_t)(2 * k + f) * R + j + 1) * P + kGhostX + i];
            }
            cs[k * 33 + u] = v;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nz * 32; e += blockDim.x) {
            const int u = e / nz, k = e - u * nz;
            const long c = c0 + u;
            if (c < ncol) dst[c * nz + k] = cs[k * 33 + u];
        }
    }
}

}  // namespace wx

using namespace wx;

extern "C" int wx_read_columns_f32(wx_ctx *c, float *T, float *q, void *stream) {
    if (!c) return WX_EINVAL;
    if (!c->fields_loaded) {
        c->err = "wx_read_columns_f32: no fields loaded";
        return WX_ESTATE;
    }
    const long ncol = (long)c->nx * c->ny;
    if (ncol == 0 || (!T && !q)) return WX_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned blocks = (unsigned)((ncol + 31) / 32);
    const size_t smem = (size_t)c->nz * 33 * sizeof(float);
    if (c->t_bytes == 4)
        columns_out_kernel<float><<<blocks, kIoThreads, smem, s>>>((const float *)c->fld[c->cur], T, q, c->nx,
                                                                   c->nz, c->P, c->R, ncol);
    else
        columns_out_kernel<double><<<blocks, kIoThreads, smem, s>>>((const double *)c->fld[c->cur], T, q, c->nx,
                                                                    c->nz, c->P, c->R, ncol);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        c->err = std::string("columns kernel: ") + cudaGetErrorString(e);
        return WX_ECUDA;
    }
    c->last_stream = s;
    return WX_OK;
}
