// wx_noalloc.cu -- FP64 mass/energy sums of a field with no allocation.
//
// For callers that cannot call cudaMalloc at all: plug-ins whose host
// application owns every device byte through its own pool and forbids other
// allocations, and real-time loops where an allocation's implicit device
// synchronisation, latency or possible failure is unacceptable.  This entry
// point takes the caller's device arrays and writes the two sums to the
// caller's device memory; the per-tile partial sums live in one file-scope
// __device__ array below instead of a buffer the library would otherwise
// allocate.
//
// Scratch facts a user needs:
//  - capacity: kMaxTiles tiles of 32 x 4 columns (1 MiB, kept by every GPU
//    that loads the library until the process exits), and at most 65535
//    tile rows (ny <= 262140); larger grids are rejected with
//    WX_EUNSUPPORTED;
//  - every call shares the array; each call overwrites every slot it reads,
//    so nothing has to start at zero, but two calls that overlap on the GPU
//    (different streams, or host threads) race on it and must be ordered by
//    the caller;
//  - the first successful call on a device looks up the array's device
//    address with cudaGetSymbolAddress while that device is current; make
//    that first call outside any stream capture.  A failed lookup is not
//    remembered: the next call tries again.
#include <mutex>

#include "wx_internal.cuh"

namespace {

constexpr int kTY = 4;
constexpr int kMaxTiles = 65536;
constexpr int kMaxTileRows = 65535;  // grid.y limit of the tile kernel
constexpr int kMaxDevices = 64;
constexpr int kLevChunk = 256;       // levels of dz staged in shared memory at a time

__device__ __align__(256) double g_partials[2 * kMaxTiles];

std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices];  // nullptr until a lookup on that device succeeded

// FP32 column sum of v * dz with dz = whi + wlo (two floats, so the FP64 dz
// is carried to about 48 bits): the product v * whi is split exactly into
// p + pe (FMA), v * wlo joins the error term, and p is added by TwoSum, so
// the FP64 total s + c is that of the FP32 values times the FP64 dz.  Every
// operation is an explicit round-to-nearest intrinsic, so the compiler can
// neither contract nor reassociate the error-free steps.
struct SumF {
    float s = 0.f, c = 0.f;
    __device__ void add(float v, float whi, float wlo) {
        const float p = __fmul_rn(v, whi);
        float pe = __fmaf_rn(v, whi, -p);
        pe = __fmaf_rn(v, wlo, pe);
        const float s1 = __fadd_rn(s, p);
        const float bp = __fsub_rn(s1, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(s1, bp)), __fsub_rn(p, bp));
        c = __fadd_rn(c, __fadd_rn(e, pe));
        s = s1;
    }
    __device__ double total() const { return (double)s + (double)c; }
};
struct SumD {
    double s = 0.0;
    __device__ void add(double v, double w, double) { s = __fma_rn(v, w, s); }
    __device__ double total() const { return s; }
};

// dz level weights in the accumulator's precision: (hi, lo) floats for FP32
// fields, (dz, 0) for FP64 fields.
template <typename T> struct Weight;
template <> struct Weight<float> {
    using W = float2;
    static __device__ W make(double d) {
        const float hi = __double2float_rn(d);
        return make_float2(hi, __double2float_rn(d - (double)hi));
    }
};
template <> struct Weight<double> {
    using W = double2;
    static __device__ W make(double d) { return make_double2(d, 0.0); }
};

template <typename T, typename Acc>
__global__ void __launch_bounds__(32 * kTY) tile_sums(const T *__restrict__ Tf, const T *__restrict__ qf,
                                                      const double *__restrict__ dz, int nx, int ny, int nz,
                                                      double *__restrict__ part) {
    using W = typename Weight<T>::W;
    __shared__ W wk[kLevChunk];
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * kTY + threadIdx.y;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const bool valid = i < nx && j < ny;
    const size_t plane = (size_t)nx * ny, col = (size_t)j * nx + i;
    Acc st, sq;
    for (int k0 = 0; k0 < nz; k0 += kLevChunk) {
        const int kn = min(kLevChunk, nz - k0);
        __syncthreads();
        for (int e = tid; e < kn; e += 32 * kTY) wk[e] = Weight<T>::make(dz[k0 + e]);
        __syncthreads();
        if (valid) {
            for (int k = 0; k < kn; ++k) {
                const W w = wk[k];
                const size_t o = (size_t)(k0 + k) * plane + col;
                st.add(Tf[o], w.x, w.y);
                sq.add(qf[o], w.x, w.y);
            }
        }
    }
    double mq = valid ? sq.total() : 0.0, mt = valid ? st.total() : 0.0;
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
    if (tid == 0) {
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

// Device address of the scratch array on the current device `dev`; looked
// up once per device and kept only when the lookup succeeded.
double *scratch_for(int dev, cudaError_t *err) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_partials);
        if (e != cudaSuccess || !p) {
            (void)cudaGetLastError();  // clear it, so that a later call can try again
            *err = e != cudaSuccess ? e : cudaErrorInvalidSymbol;
            return nullptr;
        }
        g_scratch_addr[dev] = p;
    }
    return static_cast<double *>(g_scratch_addr[dev]);
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
    if (ty > kMaxTileRows)
        return fail(WX_EUNSUPPORTED, "wx_sums_noalloc: ny exceeds 4*65535 = 262140 rows (the tile grid's row limit)");
    if (tx * ty > kMaxTiles)
        return fail(WX_EUNSUPPORTED,
                    "wx_sums_noalloc: grid needs more than 65536 tiles of 32x4 columns (the fixed scratch size)");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(WX_ECUDA, "wx_sums_noalloc: no usable current device");
    cudaError_t le = cudaSuccess;
    double *part = scratch_for(dev, &le);
    if (!part) {
        g_err = std::string("wx_sums_noalloc: cudaGetSymbolAddress of the scratch array failed: ") +
                cudaGetErrorString(le);
        return WX_ECUDA;
    }
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
