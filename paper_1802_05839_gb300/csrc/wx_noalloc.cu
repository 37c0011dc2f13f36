// wx_noalloc.cu -- FP64 mass/energy sums of a field with no allocation.
//
// For callers that cannot call cudaMalloc at all: code running inside a
// CUDA-graph capture or a pool-managed runtime that forbids device
// allocation, plug-ins whose host application owns every device byte, and
// real-time loops where an allocation's latency or failure is unacceptable.
// This entry point takes the caller's device arrays and writes the two sums
// to the caller's device memory; the per-tile partial sums live in one
// file-scope __device__ array below instead of a buffer the library would
// otherwise allocate.
//
// Scratch facts a user needs:
//  - capacity: kMaxTiles tiles of 32 x 4 columns (1 MiB, kept by every GPU
//    that loads the library until the process exits); larger grids are
//    rejected with WX_EUNSUPPORTED;
//  - every call shares the array; each call overwrites every slot it reads,
//    so nothing has to start at zero, but two calls that overlap on the GPU
//    (different streams, or host threads) race on it and must be ordered by
//    the caller;
//  - the first call on a device looks up the array's device address with
//    cudaGetSymbolAddress while that device is current; make that first
//    call outside any stream capture.
#include <mutex>

#include "wx_internal.cuh"

namespace {

constexpr int kTY = 4;
constexpr int kMaxTiles = 65536;
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_partials[2 * kMaxTiles];

void *g_scratch_addr[kMaxDevices];
std::once_flag g_scratch_once[kMaxDevices];
cudaError_t g_scratch_err[kMaxDevices];

// Column sum in the input precision (compensated in FP32), as the step kernel
// tallies its own state.
struct SumF {
    float s = 0.f, c = 0.f;
    __device__ void add(float v, float w) {
        const float p = v * w, pe = fmaf(v, w, -p);
        const float s1 = s + p, bp = s1 - s;
        c += ((s - (s1 - bp)) + (p - bp)) + pe;
        s = s1;
    }
    __device__ double total() const { return (double)s + (double)c; }
};
struct SumD {
    double s = 0.0;
    __device__ void add(double v, double w) { s = fma(v, w, s); }
    __device__ double total() const { return s; }
};

template <typename T, typename Acc>
__global__ void __launch_bounds__(32 * kTY) tile_sums(const T *__restrict__ Tf, const T *__restrict__ qf,
                                                      const double *__restrict__ dz, int nx, int ny, int nz,
                                                      double *__restrict__ part) {
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * kTY + threadIdx.y;
    double mq = 0.0, mt = 0.0;
    if (i < nx && j < ny) {
        Acc st, sq;
        const size_t plane = (size_t)nx * ny, col = (size_t)j * nx + i;
        for (int k = 0; k < nz; ++k) {
            const T w = (T)dz[k];
            st.add(Tf[k * plane + col], w);
            sq.add(qf[k * plane + col], w);
        }
        mt = st.total();
        mq = sq.total();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mq += __shfl_down_sync(0xffffffffu, mq, o);
        mt += __shfl_down_sync(0xffffffffu, mt, o);
    }
    __shared__ double red[2 * kTY];
    if (threadIdx.x == 0) {
        red[2 * threadIdx.y] = mq;
        red[2 * threadIdx.y + 1] = mt;
    }
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < kTY; ++w) {
            a += red[2 * w];
            b += red[2 * w + 1];
        }
        const size_t t = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
        part[2 * t] = a;
        part[2 * t + 1] = b;
    }
}

__global__ void __launch_bounds__(1024) finalize(const double *__restrict__ part, long ntiles, double h2,
                                                 double *__restrict__ out) {
    __shared__ double sq[1024], st[1024];
    double q = 0.0, t = 0.0;
    for (long b = threadIdx.x; b < ntiles; b += blockDim.x) {
        q += part[2 * b];
        t += part[2 * b + 1];
    }
    sq[threadIdx.x] = q;
    st[threadIdx.x] = t;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sq[threadIdx.x] += sq[threadIdx.x + o];
            st[threadIdx.x] += st[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = h2 * sq[0];
        out[1] = h2 * st[0];
    }
}

thread_local std::string g_err;

int fail(int code, const char *msg) {
    g_err = msg;
    return code;
}

}  // namespace

extern "C" const char *wx_sums_noalloc_error(void) { return g_err.c_str(); }

extern "C" int wx_sums_noalloc(const void *T, const void *q, int dtype, int nx, int ny, int nz,
                               const double *dz, double h, double *out, void *stream) {
    if (!T || !q || !dz || !out) return fail(WX_EINVAL, "wx_sums_noalloc: NULL pointer");
    if (nx < 1 || ny < 1 || nz < 1) return fail(WX_EINVAL, "wx_sums_noalloc: sizes must be >= 1");
    if (dtype != WX_F32 && dtype != WX_F64) return fail(WX_EINVAL, "wx_sums_noalloc: dtype must be WX_F32 or WX_F64");
    if (!(h > 0)) return fail(WX_EINVAL, "wx_sums_noalloc: h must be > 0");
    const long tx = (nx + 31) / 32, ty = (ny + kTY - 1) / kTY;
    if (tx * ty > kMaxTiles || ty > 65535)
        return fail(WX_EUNSUPPORTED,
                    "wx_sums_noalloc: grid needs more than 65536 tiles of 32x4 columns (the fixed scratch size)");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(WX_ECUDA, "wx_sums_noalloc: no usable current device");
    std::call_once(g_scratch_once[dev], [dev] {
        g_scratch_err[dev] = cudaGetSymbolAddress(&g_scratch_addr[dev], g_partials);
    });
    if (g_scratch_err[dev] != cudaSuccess || !g_scratch_addr[dev])
        return fail(WX_ECUDA, "wx_sums_noalloc: cudaGetSymbolAddress of the scratch array failed");
    double *part = static_cast<double *>(g_scratch_addr[dev]);
    cudaStream_t s = (cudaStream_t)stream;
    dim3 grid((unsigned)tx, (unsigned)ty), block(32, kTY);
    if (dtype == WX_F32)
        tile_sums<float, SumF><<<grid, block, 0, s>>>((const float *)T, (const float *)q, dz, nx, ny, nz, part);
    else
        tile_sums<double, SumD><<<grid, block, 0, s>>>((const double *)T, (const double *)q, dz, nx, ny, nz, part);
    finalize<<<1, 1024, 0, s>>>(part, tx * ty, h * h, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(WX_ECUDA, cudaGetErrorString(e));
    return WX_OK;
}
