// wx_mlp.cu -- BF16 tcgen05 GEMMs and the MLP surrogate of the column
// physics: forward, backward, Adam, the residual-checked surrogate step.
//
// GEMM: C[M][N] = A[M][K] . B[N][K]^T, A and B BF16 and K-major in global
// memory, FP32 accumulation in tensor memory.  A persistent kernel, one CTA
// per SM, walks the 128 x BN output tiles (n fastest, so that the CTAs
// running at the same time share each A tile in L2) with three roles:
//   warp 0 (one lane): streams 128 x 64 and BN x 64 K-slabs of A and B
//     through a shared-memory ring with TMA (128-byte swizzle);
//   warp 1 (one lane): issues tcgen05.mma (M = 128, N = BN, K = 16, four per
//     slab) into one of two TMEM accumulators, commits each slab back to its
//     ring slot and each finished tile to the epilogue;
//   warps 2..17: drain the other accumulator with tcgen05.ld and apply the
//     epilogue (bias, GELU, GELU' for backward) on the way to global memory,
//     then hand the accumulator back -- so the epilogue of tile i runs under
//     the MMAs of tile i+1.
// Every wait is bounded; a timeout sets a status bit and all roles stop.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "ptx.cuh"
#include "wx_internal.cuh"

namespace wx {

enum GemmEpi : int {
    EPI_F32 = 0,        // out_f32 = acc (+ bias)
    EPI_GELU = 1,       // z = acc + bias: out_bf16 = GELU(z), out2_bf16 = z
    EPI_DGELU = 2,      // out_bf16 = acc * GELU'(aux), aux = saved z (bf16)
    EPI_BIAS_BF16 = 3,  // out_bf16 = acc + bias
};

struct GemmArgs {
    int M, N, K;
    const float *bias;          // [N] or nullptr
    const __nv_bfloat16 *aux;   // [M][N] (EPI_DGELU)
    void *out;                  // [M][N] f32 or bf16
    __nv_bfloat16 *out2;        // [M][N] (EPI_GELU)
    unsigned *status;
};

constexpr int kGemmBK = 64;   // BF16 K per slab: one 128-byte swizzle row
constexpr int kEpiWarps = 16;  // epilogue warps: 4 per TMEM lane quarter
constexpr int kGemmThreads = 32 * (2 + kEpiWarps);
// Ring depth: 4 slots of 48 KB for 256-column tiles, 6 of 32 KB for 128.
__host__ __device__ constexpr int gemm_stages(int BN) { return BN == 256 ? 4 : 6; }
__host__ __device__ constexpr int gemm_smem(int BN) {
    return gemm_stages(BN) * (128 * kGemmBK * 2 + BN * kGemmBK * 2) + 1024 + 256;
}

// exact GELU (the erf form) and its derivative
__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    const float cdf = 0.5f * (1.f + erff(z * 0.70710678118654752f));
    const float pdf = 0.39894228040143268f * expf(-0.5f * z * z);
    return cdf + z * pdf;
}

template <int BN, int EPI>
__global__ void __launch_bounds__(kGemmThreads, 1) gemm_kernel(const __grid_constant__ CUtensorMap ta,
                                                            const __grid_constant__ CUtensorMap tb,
                                                            const GemmArgs g) {
    constexpr int BM = 128;
    constexpr int S = gemm_stages(BN);
    constexpr uint32_t A_BYTES = BM * kGemmBK * 2, B_BYTES = BN * kGemmBK * 2;
    constexpr uint32_t STAGE = A_BYTES + B_BYTES;
    constexpr int CPW = BN / 4;  // accumulator columns per epilogue warp
    extern __shared__ __align__(1024) unsigned char gsm[];
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(gsm) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(base + S * STAGE);
    uint64_t *empty = full + S;
    uint64_t *acc_full = empty + S;     // [2] MMA -> epilogue
    uint64_t *acc_empty = acc_full + 2; // [2] epilogue -> MMA
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int nk = g.K / kGemmBK, nN = g.N / BN;
    const long ntiles = (long)(g.M / BM) * nN;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], kEpiWarps);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(tmem_slot, 2 * BN);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // producer: (tile, slab) in order through the ring; a slot is
            // refilled once the MMAs that read it have completed
            prefetch_tmap(&ta);
            prefetch_tmap(&tb);
            long issued = 0;
            for (long t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
                const int m0 = (int)(t / nN) * BM, n0 = (int)(t % nN) * BN;
                for (int kb = 0; kb < nk; ++kb, ++issued) {
                    const int s = (int)(issued % S);
                    const uint32_t ph = (uint32_t)((issued / S) & 1);
                    if (*abort_flag || !mbar_wait_bounded(&empty[s], ph ^ 1u)) {
                        *abort_flag = 1;
                        break;
                    }
                    unsigned char *sa = base + s * STAGE;
                    mbar_arrive_expect_tx(&full[s], STAGE);
                    tma_load_2d(sa, &ta, &full[s], kb * kGemmBK, m0);
                    tma_load_2d(sa + A_BYTES, &tb, &full[s], kb * kGemmBK, n0);
                }
            }
            // the ring's last copies have landed before the CTA may exit
            for (long q = issued - 1; q >= 0 && q >= issued - S; --q)
                (void)mbar_wait_bounded(&full[q % S], (uint32_t)((q / S) & 1));
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(BM, BN);
            long used = 0;
            int it = 0;
            for (long t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, ++it) {
                const int b = it & 1;
                const uint32_t use = (uint32_t)(it >> 1);
                if (!mbar_wait_bounded(&acc_empty[b], (use & 1u) ^ 1u)) {
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * BN);
                bool ok = true;
                for (int kb = 0; kb < nk; ++kb, ++used) {
                    const int s = (int)(used % S);
                    if (*abort_flag || !mbar_wait_bounded(&full[s], (uint32_t)((used / S) & 1))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const unsigned char *sa = base + s * STAGE;
                    const uint64_t ad = smem_desc_sw128(sa), bd = smem_desc_sw128(sa + A_BYTES);
#pragma unroll
                    for (int kk = 0; kk < kGemmBK / 16; ++kk)
                        // +32 bytes per K = 16 step inside the 128-byte swizzle row
                        tc_mma_bf16(d, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), idesc, (kb | kk) != 0);
                    tc_commit(&empty[s]);
                }
                if (!ok) {
                    *abort_flag = 1;
                    break;
                }
                tc_commit(&acc_full[b]);  // arrives when every MMA of the tile has completed
            }
        }
    } else {
        // epilogue: warp w drains TMEM lanes 32 (w % 4) .. +31 (rows
        // m0 + 32 (w % 4) + lane), columns [CPW p, CPW (p + 1)), p = (w - 2) / 4
        const int quarter = warp & 3, part = (warp - 2) >> 2;
        int it = 0;
        for (long t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
            const int b = it & 1;
            const uint32_t use = (uint32_t)(it >> 1);
            bool ok = !*abort_flag && mbar_wait_bounded(&acc_full[b], use & 1u);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const int m0 = (int)(t / nN) * BM, n0 = (int)(t % nN) * BN;
            const int row = m0 + quarter * 32 + lane;
            const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * BN);
#pragma unroll 1
            for (int c0 = part * CPW; c0 < (part + 1) * CPW; c0 += 16) {
                float v[16];
                tmem_ld16(trow + c0, v);
                const int col = n0 + c0;
                float bias[16];
                if (g.bias) {
                    const float4 *bp = reinterpret_cast<const float4 *>(g.bias + col);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 b4 = bp[q];
                        bias[4 * q] = b4.x;
                        bias[4 * q + 1] = b4.y;
                        bias[4 * q + 2] = b4.z;
                        bias[4 * q + 3] = b4.w;
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q) bias[q] = 0.f;
                }
                const size_t o = (size_t)row * g.N + col;
                if (EPI == EPI_F32) {
                    float *out = reinterpret_cast<float *>(g.out) + o;
#pragma unroll
                    for (int q = 0; q < 16; q += 4)
                        *reinterpret_cast<float4 *>(out + q) =
                            make_float4(v[q] + bias[q], v[q + 1] + bias[q + 1], v[q + 2] + bias[q + 2],
                                        v[q + 3] + bias[q + 3]);
                } else {
                    __align__(16) __nv_bfloat162 o1[8];
                    __align__(16) __nv_bfloat162 o2[8];
                    __align__(16) __nv_bfloat16 zin[16];
                    if (EPI == EPI_DGELU) {
                        const uint4 *zp = reinterpret_cast<const uint4 *>(g.aux + o);
                        *reinterpret_cast<uint4 *>(zin) = zp[0];
                        *reinterpret_cast<uint4 *>(zin + 8) = zp[1];
                    }
#pragma unroll
                    for (int q = 0; q < 16; q += 2) {
                        if (EPI == EPI_GELU) {
                            const float z0 = v[q] + bias[q], z1 = v[q + 1] + bias[q + 1];
                            o1[q / 2] = __floats2bfloat162_rn(gelu(z0), gelu(z1));
                            o2[q / 2] = __floats2bfloat162_rn(z0, z1);
                        } else if (EPI == EPI_DGELU) {
                            o1[q / 2] = __floats2bfloat162_rn(v[q] * gelu_grad(__bfloat162float(zin[q])),
                                                              v[q + 1] * gelu_grad(__bfloat162float(zin[q + 1])));
                        } else {
                            o1[q / 2] = __floats2bfloat162_rn(v[q] + bias[q], v[q + 1] + bias[q + 1]);
                        }
                    }
                    __nv_bfloat16 *out = reinterpret_cast<__nv_bfloat16 *>(g.out) + o;
                    reinterpret_cast<uint4 *>(out)[0] = *reinterpret_cast<uint4 *>(o1);
                    reinterpret_cast<uint4 *>(out)[1] = *reinterpret_cast<uint4 *>(o1 + 4);
                    if (EPI == EPI_GELU && g.out2) {
                        __nv_bfloat16 *out2 = g.out2 + o;
                        reinterpret_cast<uint4 *>(out2)[0] = *reinterpret_cast<uint4 *>(o2);
                        reinterpret_cast<uint4 *>(out2)[1] = *reinterpret_cast<uint4 *>(o2 + 4);
                    }
                }
            }
            // the accumulator may be overwritten once every warp's loads are done
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) atomicOr(g.status, ST_TIMEOUT);
    if (warp == 0) tmem_dealloc(tmem, 2 * BN);
}

// ------------------------------------------------------------ launcher
static PFN_cuTensorMapEncodeTiled_v12000 encoder() {
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

// 2D BF16 row-major [rows][K] operand, box 64 (K) x box_rows, 128-byte swizzle.
static bool encode_operand(CUtensorMap *m, const void *ptr, int rows, int K, int box_rows) {
    auto enc = encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    cuuint32_t box[2] = {(cuuint32_t)kGemmBK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Descriptors are cached per (device, pointer, shape): the MLP reuses its
// buffers.  The cache is cleared when it grows past kMapCacheMax entries
// (callers that pass a fresh buffer every call, e.g. gathered minibatches).
constexpr size_t kMapCacheMax = 4096;
static std::mutex g_map_mu;
static std::map<std::tuple<int, const void *, int, int, int>, CUtensorMap> g_maps;

static bool operand_map(CUtensorMap *m, const void *ptr, int rows, int K, int box_rows) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_map_mu);
    auto key = std::make_tuple(dev, ptr, rows, K, box_rows);
    auto it = g_maps.find(key);
    if (it != g_maps.end()) {
        *m = it->second;
        return true;
    }
    if (!encode_operand(m, ptr, rows, K, box_rows)) return false;
    if (g_maps.size() >= kMapCacheMax) g_maps.clear();
    g_maps[key] = *m;
    return true;
}

template <int BN, int EPI> static cudaError_t gemm_launch(const CUtensorMap &a, const CUtensorMap &b, const GemmArgs &g,
                                                         cudaStream_t s) {
    auto k = gemm_kernel<BN, EPI>;
    const int smem = gemm_smem(BN);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long tiles = (long)(g.M / 128) * (g.N / BN);
    k<<<(unsigned)std::min<long>(tiles, sms), kGemmThreads, smem, s>>>(a, b, g);
    return cudaGetLastError();
}

// C = A . B^T with the epilogue `epi`.  M % 128 == 0, K % 64 == 0, N % 128
// == 0 (tiles of 256 columns when N % 256 == 0).
int gemm(const void *A, const void *B, int M, int N, int K, int epi, const float *bias, const void *aux, void *out,
         void *out2, unsigned *status, cudaStream_t s, std::string &err) {
    if (M <= 0 || N <= 0 || K <= 0 || M % 128 || N % 128 || K % kGemmBK) {
        err = "gemm: M and N must be multiples of 128 and K of 64";
        return WX_EINVAL;
    }
    const int BN = (N % 256 == 0) ? 256 : 128;
    CUtensorMap ta, tb;
    if (!operand_map(&ta, A, M, K, 128) || !operand_map(&tb, B, N, K, BN)) {
        err = "gemm: tensor map encoding failed (alignment?)";
        return WX_ECUDA;
    }
    GemmArgs g{M, N, K, bias, reinterpret_cast<const __nv_bfloat16 *>(aux), out,
               reinterpret_cast<__nv_bfloat16 *>(out2), status};
    cudaError_t e = cudaErrorInvalidValue;
#define WX_GEMM_CASE(E)                                                                        \
    case E:                                                                                    \
        e = (BN == 256) ? gemm_launch<256, E>(ta, tb, g, s) : gemm_launch<128, E>(ta, tb, g, s); \
        break;
    switch (epi) {
        WX_GEMM_CASE(EPI_F32)
        WX_GEMM_CASE(EPI_GELU)
        WX_GEMM_CASE(EPI_DGELU)
        WX_GEMM_CASE(EPI_BIAS_BF16)
        default: err = "gemm: unknown epilogue"; return WX_EINVAL;
    }
#undef WX_GEMM_CASE
    if (e != cudaSuccess) {
        err = std::string("gemm: ") + cudaGetErrorString(e);
        return WX_ECUDA;
    }
    return WX_OK;
}

}  // namespace wx

using namespace wx;

static thread_local std::string g_mlp_err;

extern "C" const char *wx_mlp_last_error(void) { return g_mlp_err.c_str(); }

extern "C" int wx_gemm_bf16(const void *A, const void *B, int M, int N, int K, int epilogue, const float *bias,
                            const void *aux, void *out, void *out2, unsigned *status, void *stream) {
    if (!A || !B || !out || !status) {
        g_mlp_err = "wx_gemm_bf16: NULL pointer";
        return WX_EINVAL;
    }
    if ((epilogue == EPI_GELU && !bias) || (epilogue == EPI_DGELU && !aux)) {
        g_mlp_err = "wx_gemm_bf16: epilogue needs bias/out2 (GELU) or aux (GELU')";
        return WX_EINVAL;
    }
    return gemm(A, B, M, N, K, epilogue, bias, aux, out, out2, status, (cudaStream_t)stream, g_mlp_err);
}

// =====================================================================
// MLP surrogate of the column physics
//   x (232 = T*, q*, kappa_v, alpha dz per level; normalised, padded to 256)
//   -> 512 -> 512 -> 512 (GELU) -> 116 (dt-free tendencies H and vdiff rate,
//   normalised, padded to 128)
// =====================================================================
namespace wx {

constexpr int kNZ = 58, kIn = 4 * kNZ, kInP = 256, kHid = 512, kOut = 2 * kNZ, kOutP = 128;
// Input rows carry each normalised feature as a two-term BF16 expansion
// x ~ hi + lo (hi = bf16(x), lo = bf16(x - hi)): [hi (256) | lo (256)].  The
// first layer multiplies both halves by the same weights, so its products
// see the input to ~16 significant bits instead of BF16's 8.
constexpr int kXW = 2 * kInP;
constexpr int kLayers = 4;
__host__ __device__ constexpr int layer_in(int l) { return l == 0 ? kInP : kHid; }
// K of the layer's forward GEMM (the first layer runs over both halves)
__host__ __device__ constexpr int layer_k(int l) { return l == 0 ? kXW : kHid; }
__host__ __device__ constexpr int layer_out(int l) { return l == 3 ? kOutP : kHid; }

}  // namespace wx

struct wx_mlp {
    int max_batch = 0;
    float *W[wx::kLayers] = {}, *b[wx::kLayers] = {};          // FP32 master [N][K], [N]
    __nv_bfloat16 *Wb[wx::kLayers] = {}, *WbT[wx::kLayers] = {};  // BF16 [N][K] and [K][N]
    float *mW[wx::kLayers] = {}, *vW[wx::kLayers] = {}, *mb[wx::kLayers] = {}, *vb[wx::kLayers] = {};
    float *dW[wx::kLayers] = {}, *db[wx::kLayers] = {};
    float *norm = nullptr;   // [4][kIn | kOut]: mean_in, std_in, mean_out, std_out (padded to 256)
    float *lev = nullptr;    // [2][kNZ]: kappa_lev, alpha*dz (feature inputs)
    // activations for batch rows
    __nv_bfloat16 *X = nullptr, *Z[3] = {}, *H[3] = {}, *dY = nullptr, *dZ[3] = {}, *TA = nullptr, *TB = nullptr;
    float *Y = nullptr, *loss = nullptr;
    unsigned *status = nullptr;
    long adam_t = 0;
    std::string err;
};

namespace wx {

// ------------------------------------------------------------ small kernels
__global__ void transpose_bf16_kernel(const __nv_bfloat16 *__restrict__ in, __nv_bfloat16 *__restrict__ out,
                                      int rows, int cols, int ld) {
    __shared__ __nv_bfloat16 t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int r = r0 + y, c = c0 + threadIdx.x;
        if (r < rows && c < cols) t[y][threadIdx.x] = in[(size_t)r * ld + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int c = c0 + y, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[(size_t)c * rows + r] = t[threadIdx.x][y];
    }
}

// db[n] = sum_m dZT[n][m], one block per row, fixed-order tree.
__global__ void rowsum_bf16_kernel(const __nv_bfloat16 *__restrict__ in, int cols, float *__restrict__ out) {
    __shared__ float red[256];
    const int r = blockIdx.x;
    float s = 0.f;
    for (int c = threadIdx.x; c < cols; c += blockDim.x) s += __bfloat162float(in[(size_t)r * cols + c]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[r] = red[0];
}

// dY = 2 (Y - Yt) / (M * kOut) on the kOut real outputs (bf16), 0 on the
// padding; per-block squared-error partials for the loss.
__global__ void mse_grad_kernel(const float *__restrict__ Y, const float *__restrict__ Yt, int M,
                                __nv_bfloat16 *__restrict__ dY, float *__restrict__ part) {
    __shared__ float red[256];
    float s = 0.f;
    const size_t n = (size_t)M * kOutP;
    const float scale = 2.f / ((float)M * kOut);
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % kOutP);
        float g = 0.f;
        if (c < kOut) {
            const float d = Y[e] - Yt[e];
            s += d * d;
            g = scale * d;
        }
        dY[e] = __float2bfloat16_rn(g);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void loss_finalize_kernel(const float *__restrict__ part, int n, int M, float *__restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    out[0] = (float)(s / ((double)M * kOut));
}

// BF16 copies of master element e = (n, k) of an [N][K] matrix: pb [N][K],
// or [N][2K] with the row written twice for the first layer (dup); pbT
// [K][N] (feeds the input-gradient GEMM) unless NULL.
__device__ __forceinline__ void store_copies(float v, long e, int N, int K, int dup, __nv_bfloat16 *pb,
                                             __nv_bfloat16 *pbT) {
    const __nv_bfloat16 q = __float2bfloat16_rn(v);
    const int nn = (int)(e / K), kk = (int)(e % K);
    if (dup) {
        pb[(size_t)nn * 2 * K + kk] = q;
        pb[(size_t)nn * 2 * K + K + kk] = q;
    } else {
        pb[e] = q;
    }
    if (pbT) pbT[(size_t)kk * N + nn] = q;
}

// Adam (beta1, beta2, eps) on FP32 masters, then the BF16 copies.
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, long n, int N, int K, float lr, float b1, float b2, float eps,
                            float c1, float c2, int dup, __nv_bfloat16 *__restrict__ pb,
                            __nv_bfloat16 *__restrict__ pbT) {
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const float gi = g[e];
        const float mi = b1 * m[e] + (1.f - b1) * gi;
        const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
        m[e] = mi;
        v[e] = vi;
        const float pi = p[e] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[e] = pi;
        if (pb) store_copies(pi, e, N, K, dup, pb, pbT);
    }
}

__global__ void to_bf16_kernel(const float *__restrict__ p, long n, int N, int K, int dup,
                               __nv_bfloat16 *__restrict__ pb, __nv_bfloat16 *__restrict__ pbT) {
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
        store_copies(p[e], e, N, K, dup, pb, pbT);
}

// Features of ncol columns given as [ncol][nz] arrays (T*, q*), kappa_mult
// per column (NULL = 1): normalised BF16 rows [ncol_pad][256].
__global__ void features_cols_kernel(const float *__restrict__ Ts, const float *__restrict__ qs,
                                     const float *__restrict__ km, long ncol, long ncol_pad,
                                     const float *__restrict__ lev, const float *__restrict__ norm,
                                     __nv_bfloat16 *__restrict__ X) {
    const long col = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncol_pad) return;
    __nv_bfloat16 *row = X + col * kXW;
    if (col >= ncol) {
        for (int f = 0; f < kXW; ++f) row[f] = __float2bfloat16_rn(0.f);
        return;
    }
    const float s = km ? km[col] : 1.f;
    for (int f = 0; f < kInP; ++f) {
        float x = 0.f;
        if (f < kIn) {
            const int k = f % kNZ, kind = f / kNZ;
            const float raw = kind == 0 ? Ts[col * kNZ + k]
                              : kind == 1 ? qs[col * kNZ + k]
                              : kind == 2 ? s * lev[k]
                                          : lev[kNZ + k];
            x = (raw - norm[f]) * (1.f / norm[kInP + f]);
        }
        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
        row[f] = hi;
        row[kInP + f] = __float2bfloat16_rn(x - __bfloat162float(hi));
    }
}

// Targets from tend [ncol][2][nz] = (H_k, vdiff_k): normalised FP32 rows
// [ncol_pad][128] (zeros past the data and on the padding columns).
__global__ void targets_kernel(const float *__restrict__ tend, long ncol, long ncol_pad,
                               const float *__restrict__ norm, float *__restrict__ Yt) {
    const long col = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncol_pad) return;
    const float *mo = norm + 2 * kInP, *so = norm + 3 * kInP;
    for (int c = 0; c < kOutP; ++c) {
        float y = 0.f;
        if (c < kOut && col < ncol) y = (tend[col * kOut + c] - mo[c]) / so[c];
        Yt[col * kOutP + c] = y;
    }
}

// Per-feature mean and standard deviation over rows of raw features, in
// FP64, fixed order (one block per feature).
__global__ void feature_stats_kernel(const float *__restrict__ Ts, const float *__restrict__ qs,
                                     const float *__restrict__ km, const float *__restrict__ tend, long ncol,
                                     const float *__restrict__ lev, float *__restrict__ norm) {
    __shared__ double s1[256], s2[256];
    const int f = blockIdx.x;  // 0..kIn-1 inputs, kIn..kIn+kOut-1 targets
    double a = 0.0, b = 0.0;
    for (long c = threadIdx.x; c < ncol; c += blockDim.x) {
        float raw;
        if (f < kIn) {
            const int k = f % kNZ, kind = f / kNZ;
            raw = kind == 0 ? Ts[c * kNZ + k]
                  : kind == 1 ? qs[c * kNZ + k]
                  : kind == 2 ? (km ? km[c] : 1.f) * lev[k]
                              : lev[kNZ + k];
        } else {
            raw = tend[c * kOut + (f - kIn)];
        }
        a += raw;
        b += (double)raw * raw;
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            s1[threadIdx.x] += s1[threadIdx.x + o];
            s2[threadIdx.x] += s2[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mean = s1[0] / (double)ncol;
        const double var = fmax(s2[0] / (double)ncol - mean * mean, 0.0);
        const float sd = (float)fmax(sqrt(var), 1e-6 * fmax(fabs(mean), 1e-12));
        if (f < kIn) {
            norm[f] = (float)mean;
            norm[kInP + f] = sd > 0 ? sd : 1.f;
        } else {
            norm[2 * kInP + f - kIn] = (float)mean;
            norm[3 * kInP + f - kIn] = sd > 0 ? sd : 1.f;
        }
    }
}

static int grid1(long n, int t = 256) { return (int)std::min<long>(std::max<long>((n + t - 1) / t, 1), 65535L * 16); }

}  // namespace wx

// ------------------------------------------------------------ C ABI
static int mfail(wx_mlp *m, int code, const std::string &msg) {
    g_mlp_err = msg;
    if (m) m->err = msg;
    return code;
}

#define MCK(call, what)                                                                         \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return mfail(m, WX_ECUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
    } while (0)

extern "C" void wx_mlp_destroy(wx_mlp *m) {
    if (!m) return;
    for (int l = 0; l < kLayers; ++l)
        for (void *p : {(void *)m->W[l], (void *)m->b[l], (void *)m->Wb[l], (void *)m->WbT[l], (void *)m->mW[l],
                        (void *)m->vW[l], (void *)m->mb[l], (void *)m->vb[l], (void *)m->dW[l], (void *)m->db[l]})
            if (p) cudaFree(p);
    for (int i = 0; i < 3; ++i)
        for (void *p : {(void *)m->Z[i], (void *)m->H[i], (void *)m->dZ[i]})
            if (p) cudaFree(p);
    for (void *p : {(void *)m->norm, (void *)m->lev, (void *)m->X, (void *)m->dY, (void *)m->TA, (void *)m->TB,
                    (void *)m->Y, (void *)m->loss, (void *)m->status})
        if (p) cudaFree(p);
    delete m;
}

extern "C" int wx_mlp_create(int max_batch, wx_mlp **out) {
    if (!out) return mfail(nullptr, WX_EINVAL, "wx_mlp_create: out is NULL");
    *out = nullptr;
    if (max_batch < 128 || max_batch % 128) return mfail(nullptr, WX_EINVAL, "wx_mlp_create: max_batch % 128 != 0");
    wx_mlp *m = new (std::nothrow) wx_mlp();
    if (!m) return mfail(nullptr, WX_ENOMEM, "wx_mlp_create: host allocation");
    m->max_batch = max_batch;
    auto alloc = [&](void **p, size_t bytes) {
        if (cudaMalloc(p, bytes) != cudaSuccess) return false;
        return cudaMemset(*p, 0, bytes) == cudaSuccess;
    };
    bool ok = true;
    for (int l = 0; l < kLayers && ok; ++l) {
        const size_t nk = (size_t)layer_out(l) * layer_in(l), n = layer_out(l);
        ok = alloc((void **)&m->W[l], nk * 4) && alloc((void **)&m->b[l], n * 4) &&
             alloc((void **)&m->Wb[l], (size_t)layer_out(l) * layer_k(l) * 2) &&
             alloc((void **)&m->WbT[l], nk * 2) &&
             alloc((void **)&m->mW[l], nk * 4) && alloc((void **)&m->vW[l], nk * 4) &&
             alloc((void **)&m->mb[l], n * 4) && alloc((void **)&m->vb[l], n * 4) &&
             alloc((void **)&m->dW[l], nk * 4) && alloc((void **)&m->db[l], n * 4);
    }
    const size_t B = max_batch;
    for (int i = 0; i < 3 && ok; ++i)
        ok = alloc((void **)&m->Z[i], B * kHid * 2) && alloc((void **)&m->H[i], B * kHid * 2) &&
             alloc((void **)&m->dZ[i], B * kHid * 2);
    ok = ok && alloc((void **)&m->norm, 4 * kInP * 4) && alloc((void **)&m->lev, 2 * kNZ * 4) &&
         alloc((void **)&m->X, B * kXW * 2) && alloc((void **)&m->dY, B * kOutP * 2) &&
         alloc((void **)&m->TA, B * kHid * 2) && alloc((void **)&m->TB, B * kHid * 2) &&
         alloc((void **)&m->Y, B * kOutP * 4) && alloc((void **)&m->loss, 1024 * 4) &&
         alloc((void **)&m->status, sizeof(unsigned));
    if (!ok) {
        cudaGetLastError();
        wx_mlp_destroy(m);
        return mfail(nullptr, WX_ENOMEM, "wx_mlp_create: device allocation failed");
    }
    // unit normalisation until set
    std::vector<float> nrm(4 * kInP, 0.f);
    for (int i = 0; i < kInP; ++i) nrm[kInP + i] = nrm[3 * kInP + i] = 1.f;
    cudaMemcpy(m->norm, nrm.data(), nrm.size() * 4, cudaMemcpyHostToDevice);
    *out = m;
    return WX_OK;
}

// Weights from host FP32 arrays W_l [out][in] (real sizes 512x232, 512x512,
// 512x512, 116x512) and biases b_l [out]; zero-padded on the device.
extern "C" int wx_mlp_set_weights(wx_mlp *m, const float *const *W, const float *const *b) {
    if (!m || !W || !b) return mfail(m, WX_EINVAL, "wx_mlp_set_weights: NULL");
    const int real_in[kLayers] = {kIn, kHid, kHid, kHid}, real_out[kLayers] = {kHid, kHid, kHid, kOut};
    for (int l = 0; l < kLayers; ++l) {
        const int N = layer_out(l), K = layer_in(l);
        std::vector<float> w((size_t)N * K, 0.f), bb(N, 0.f);
        for (int n = 0; n < real_out[l]; ++n) {
            for (int k = 0; k < real_in[l]; ++k) w[(size_t)n * K + k] = W[l][(size_t)n * real_in[l] + k];
            bb[n] = b[l][n];
        }
        MCK(cudaMemcpy(m->W[l], w.data(), w.size() * 4, cudaMemcpyHostToDevice), "upload W");
        MCK(cudaMemcpy(m->b[l], bb.data(), bb.size() * 4, cudaMemcpyHostToDevice), "upload b");
        MCK(cudaMemset(m->mW[l], 0, w.size() * 4), "reset Adam");
        MCK(cudaMemset(m->vW[l], 0, w.size() * 4), "reset Adam");
        MCK(cudaMemset(m->mb[l], 0, bb.size() * 4), "reset Adam");
        MCK(cudaMemset(m->vb[l], 0, bb.size() * 4), "reset Adam");
        to_bf16_kernel<<<grid1((long)N * K), 256>>>(m->W[l], (long)N * K, N, K, l == 0, m->Wb[l],
                                                     l == 0 ? nullptr : m->WbT[l]);
    }
    m->adam_t = 0;
    MCK(cudaDeviceSynchronize(), "wx_mlp_set_weights");
    return WX_OK;
}

extern "C" int wx_mlp_get_weights(wx_mlp *m, float *const *W, float *const *b) {
    if (!m || !W || !b) return mfail(m, WX_EINVAL, "wx_mlp_get_weights: NULL");
    const int real_in[kLayers] = {kIn, kHid, kHid, kHid}, real_out[kLayers] = {kHid, kHid, kHid, kOut};
    MCK(cudaDeviceSynchronize(), "wx_mlp_get_weights");
    for (int l = 0; l < kLayers; ++l) {
        const int N = layer_out(l), K = layer_in(l);
        std::vector<float> w((size_t)N * K), bb(N);
        MCK(cudaMemcpy(w.data(), m->W[l], w.size() * 4, cudaMemcpyDeviceToHost), "download W");
        MCK(cudaMemcpy(bb.data(), m->b[l], bb.size() * 4, cudaMemcpyDeviceToHost), "download b");
        for (int n = 0; n < real_out[l]; ++n) {
            for (int k = 0; k < real_in[l]; ++k) W[l][(size_t)n * real_in[l] + k] = w[(size_t)n * K + k];
            b[l][n] = bb[n];
        }
    }
    return WX_OK;
}

// Gradients (FP32) of the last training step, same layout as the weights.
extern "C" int wx_mlp_get_grads(wx_mlp *m, float *const *dW, float *const *db) {
    if (!m || !dW || !db) return mfail(m, WX_EINVAL, "wx_mlp_get_grads: NULL");
    const int real_in[kLayers] = {kIn, kHid, kHid, kHid}, real_out[kLayers] = {kHid, kHid, kHid, kOut};
    MCK(cudaDeviceSynchronize(), "wx_mlp_get_grads");
    for (int l = 0; l < kLayers; ++l) {
        const int N = layer_out(l), K = layer_in(l);
        std::vector<float> w((size_t)N * K), bb(N);
        MCK(cudaMemcpy(w.data(), m->dW[l], w.size() * 4, cudaMemcpyDeviceToHost), "download dW");
        MCK(cudaMemcpy(bb.data(), m->db[l], bb.size() * 4, cudaMemcpyDeviceToHost), "download db");
        for (int n = 0; n < real_out[l]; ++n) {
            for (int k = 0; k < real_in[l]; ++k) dW[l][(size_t)n * real_in[l] + k] = w[(size_t)n * K + k];
            db[l][n] = bb[n];
        }
    }
    return WX_OK;
}

// Normalisation (host arrays): mean_in[232], std_in[232], mean_out[116],
// std_out[116]; per-level feature inputs kappa_lev[58], alpha*dz[58].
extern "C" int wx_mlp_set_norm(wx_mlp *m, const float *mean_in, const float *std_in, const float *mean_out,
                               const float *std_out) {
    if (!m || !mean_in || !std_in || !mean_out || !std_out) return mfail(m, WX_EINVAL, "wx_mlp_set_norm: NULL");
    std::vector<float> nrm(4 * kInP, 0.f);
    for (int i = 0; i < kInP; ++i) nrm[kInP + i] = nrm[3 * kInP + i] = 1.f;
    for (int i = 0; i < kIn; ++i) {
        nrm[i] = mean_in[i];
        nrm[kInP + i] = std_in[i];
    }
    for (int i = 0; i < kOut; ++i) {
        nrm[2 * kInP + i] = mean_out[i];
        nrm[3 * kInP + i] = std_out[i];
    }
    MCK(cudaMemcpy(m->norm, nrm.data(), nrm.size() * 4, cudaMemcpyHostToDevice), "upload norm");
    return WX_OK;
}

extern "C" int wx_mlp_get_norm(wx_mlp *m, float *mean_in, float *std_in, float *mean_out, float *std_out) {
    if (!m) return mfail(m, WX_EINVAL, "wx_mlp_get_norm: NULL");
    std::vector<float> nrm(4 * kInP);
    MCK(cudaMemcpy(nrm.data(), m->norm, nrm.size() * 4, cudaMemcpyDeviceToHost), "download norm");
    for (int i = 0; i < kIn; ++i) {
        if (mean_in) mean_in[i] = nrm[i];
        if (std_in) std_in[i] = nrm[kInP + i];
    }
    for (int i = 0; i < kOut; ++i) {
        if (mean_out) mean_out[i] = nrm[2 * kInP + i];
        if (std_out) std_out[i] = nrm[3 * kInP + i];
    }
    return WX_OK;
}

extern "C" int wx_mlp_set_levels(wx_mlp *m, int nz, const float *kappa_lev, const float *alpha_dz) {
    if (!m || !kappa_lev || !alpha_dz) return mfail(m, WX_EINVAL, "wx_mlp_set_levels: NULL");
    if (nz != kNZ) return mfail(m, WX_EUNSUPPORTED, "wx_mlp_set_levels: the surrogate is built for 58 levels");
    MCK(cudaMemcpy(m->lev, kappa_lev, kNZ * 4, cudaMemcpyHostToDevice), "upload levels");
    MCK(cudaMemcpy(m->lev + kNZ, alpha_dz, kNZ * 4, cudaMemcpyHostToDevice), "upload levels");
    return WX_OK;
}

// Statistics of a training set (device arrays [ncol][58] T*, q*, kappa_mult
// [ncol] or NULL, tend [ncol][2][58]) -> the normalisation (FP64 sums).
extern "C" int wx_mlp_fit_norm(wx_mlp *m, const float *Ts, const float *qs, const float *km, const float *tend,
                               long ncol, void *stream) {
    if (!m || !Ts || !qs || !tend || ncol <= 0) return mfail(m, WX_EINVAL, "wx_mlp_fit_norm: bad arguments");
    feature_stats_kernel<<<kIn + kOut, 256, 0, (cudaStream_t)stream>>>(Ts, qs, km, tend, ncol, m->lev, m->norm);
    MCK(cudaGetLastError(), "feature stats kernel");
    return WX_OK;
}

// Normalised BF16 features [ncol_pad][256] and FP32 targets [ncol_pad][128]
// (tend may be NULL) of device columns; ncol_pad = ncol rounded up to 128.
extern "C" int wx_mlp_prepare(wx_mlp *m, const float *Ts, const float *qs, const float *km, const float *tend,
                              long ncol, void *X, float *Yt, void *stream) {
    if (!m || !Ts || !qs || !X || ncol < 0) return mfail(m, WX_EINVAL, "wx_mlp_prepare: bad arguments");
    const long pad = (ncol + 127) / 128 * 128;
    cudaStream_t s = (cudaStream_t)stream;
    features_cols_kernel<<<grid1(pad, 128), 128, 0, s>>>(Ts, qs, km, ncol, pad, m->lev, m->norm,
                                                         reinterpret_cast<__nv_bfloat16 *>(X));
    if (tend && Yt) targets_kernel<<<grid1(pad, 128), 128, 0, s>>>(tend, ncol, pad, m->norm, Yt);
    MCK(cudaGetLastError(), "prepare kernels");
    return WX_OK;
}

namespace wx {
// Forward pass of M rows (M % 128 == 0, <= max_batch) from BF16 rows X
// [M][512] (hi | lo); Z/H kept for backward; normalised outputs in m->Y
// [M][128] (or `Yout`).
static int mlp_forward(wx_mlp *m, const __nv_bfloat16 *X, int M, float *Yout, cudaStream_t s,
                       bool keep_z = true) {
    const __nv_bfloat16 *in = X;
    for (int l = 0; l < 3; ++l) {
        const int rc = gemm(in, m->Wb[l], M, kHid, layer_k(l), EPI_GELU, m->b[l], nullptr, m->H[l],
                            keep_z ? m->Z[l] : nullptr, m->status, s, m->err);
        if (rc != WX_OK) return rc;
        in = m->H[l];
    }
    return gemm(in, m->Wb[3], M, kOutP, kHid, EPI_F32, m->b[3], nullptr, Yout ? Yout : m->Y, nullptr, m->status, s,
                m->err);
}

static void transpose(const __nv_bfloat16 *in, __nv_bfloat16 *out, int rows, int cols, int ld, cudaStream_t s) {
    dim3 grid((cols + 31) / 32, (rows + 31) / 32), block(32, 8);
    transpose_bf16_kernel<<<grid, block, 0, s>>>(in, out, rows, cols, ld);
}

// Loss gradient and backward pass after mlp_forward of the same rows:
//   dW_l = dZ_l^T . a_l (GEMM over the M rows of the transposed operands),
//   db_l = column sums of dZ_l,
//   dZ_{l-1} = (dZ_l . W_l) * GELU'(Z_{l-1}) (GEMM with the GELU' epilogue).
// The first layer's weight gradient takes the leading BF16 term of its
// inputs (the hi half of X).
static int mlp_backward(wx_mlp *m, const __nv_bfloat16 *X, const float *Yt, int M, float *loss, cudaStream_t s) {
    const int nblk = 256;
    mse_grad_kernel<<<nblk, 256, 0, s>>>(m->Y, Yt, M, m->dY, m->loss + 1);
    if (loss) loss_finalize_kernel<<<1, 32, 0, s>>>(m->loss + 1, nblk, M, loss);
    const __nv_bfloat16 *dout = m->dY;
    int nout = kOutP;
    for (int l = 3; l >= 0; --l) {
        const int K = layer_in(l);
        const __nv_bfloat16 *act = l == 0 ? X : m->H[l - 1];
        transpose(dout, m->TA, M, nout, nout, s);              // [nout][M]
        transpose(act, m->TB, M, K, l == 0 ? kXW : K, s);      // [K][M]
        int rc = gemm(m->TA, m->TB, nout, K, M, EPI_F32, nullptr, nullptr, m->dW[l], nullptr, m->status, s, m->err);
        if (rc != WX_OK) return rc;
        rowsum_bf16_kernel<<<nout, 256, 0, s>>>(m->TA, M, m->db[l]);
        if (l > 0) {
            rc = gemm(dout, m->WbT[l], M, K, nout, EPI_DGELU, nullptr, m->Z[l - 1], m->dZ[l - 1], nullptr,
                      m->status, s, m->err);
            if (rc != WX_OK) return rc;
            dout = m->dZ[l - 1];
            nout = kHid;
        }
    }
    return WX_OK;
}
}  // namespace wx

namespace wx {
template <typename S, typename D>
__global__ void convert_any_kernel(const S *__restrict__ src, D *__restrict__ dst, long n) {
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
        dst[e] = (D)src[e];
}

// Rows of 16-byte words: dst row r = src row idx[r] (a zero row where the
// index is outside [0, src_rows)).
__global__ void gather_rows_kernel(const uint4 *__restrict__ src, long src_rows, long words,
                                   const int *__restrict__ idx, long n, uint4 *__restrict__ dst) {
    const long total = n * words;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const long r = e / words, w = e - r * words;
        const long sr = idx[r];
        dst[e] = (sr >= 0 && sr < src_rows) ? src[sr * words + w] : make_uint4(0u, 0u, 0u, 0u);
    }
}

// Physical-unit outputs out[r][o] = Y[r][o] std_out[o] + mean_out[o], o < kOut.
__global__ void denormalize_kernel(const float *__restrict__ Y, const float *__restrict__ norm, long M,
                                   float *__restrict__ out) {
    const long total = M * kOut;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const long r = e / kOut;
        const int o = (int)(e - r * kOut);
        out[e] = fmaf(Y[r * kOutP + o], norm[3 * kInP + o], norm[2 * kInP + o]);
    }
}

static unsigned grid_of(long n) {
    const long b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 65535 * 4 ? 65535 * 4 : b));
}
}  // namespace wx

extern "C" int wx_convert(const void *src, void *dst, long n, int to_f64, void *stream) {
    if (n < 0 || (n > 0 && (!src || !dst))) return mfail(nullptr, WX_EINVAL, "wx_convert: bad arguments");
    if (n == 0) return WX_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (to_f64)
        convert_any_kernel<float, double><<<grid_of(n), 256, 0, s>>>((const float *)src, (double *)dst, n);
    else
        convert_any_kernel<double, float><<<grid_of(n), 256, 0, s>>>((const double *)src, (float *)dst, n);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? WX_OK : mfail(nullptr, WX_ECUDA, std::string("wx_convert: ") + cudaGetErrorString(e));
}

extern "C" int wx_gather_rows(const void *src, long src_rows, long row_bytes, const int *idx, long n, void *dst,
                              void *stream) {
    if (n < 0 || src_rows < 0 || row_bytes <= 0 || row_bytes % 16 || (n > 0 && (!src || !idx || !dst)) ||
        (reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) % 16)
        return mfail(nullptr, WX_EINVAL, "wx_gather_rows: rows of a multiple of 16 bytes, 16-byte aligned arrays");
    if (n == 0) return WX_OK;
    const long words = row_bytes / 16;
    gather_rows_kernel<<<grid_of(n * words), 256, 0, (cudaStream_t)stream>>>(
        (const uint4 *)src, src_rows, words, idx, n, (uint4 *)dst);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? WX_OK
                            : mfail(nullptr, WX_ECUDA, std::string("wx_gather_rows: ") + cudaGetErrorString(e));
}

// The training driver's minibatch order (host only): Fisher-Yates from the
// top with splitmix64 (Steele, Lea and Flood 2014), each draw in [0, i]
// taken as the high half of u * (i + 1) (Lemire's multiply-shift).
extern "C" int wx_permutation(long n, unsigned long long seed, int *out) {
    if (n < 0 || n > 2147483647L || (n > 0 && !out)) return WX_EINVAL;
    for (long i = 0; i < n; ++i) out[i] = (int)i;
    unsigned long long state = seed;
    auto next = [&]() {
        unsigned long long z = (state += 0x9e3779b97f4a7c15ull);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        return z ^ (z >> 31);
    };
    for (long i = n - 1; i > 0; --i) {
        const long r = (long)(((unsigned __int128)next() * (unsigned long long)(i + 1)) >> 64);
        const int t = out[i];
        out[i] = out[r];
        out[r] = t;
    }
    return WX_OK;
}

extern "C" int wx_mlp_denormalize(wx_mlp *m, const float *Y, long M, float *out, void *stream) {
    if (!m) return mfail(nullptr, WX_EINVAL, "wx_mlp_denormalize: no network");
    if (M < 0 || (M > 0 && (!Y || !out))) return mfail(m, WX_EINVAL, "wx_mlp_denormalize: bad arguments");
    if (M == 0) return WX_OK;
    denormalize_kernel<<<grid_of(M * kOut), 256, 0, (cudaStream_t)stream>>>(Y, m->norm, M, out);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? WX_OK : mfail(m, WX_ECUDA, std::string("wx_mlp_denormalize: ") + cudaGetErrorString(e));
}

extern "C" int wx_mlp_forward(wx_mlp *m, const void *X, int M, float *Y, void *stream) {
    if (!m || !X || !Y) return mfail(m, WX_EINVAL, "wx_mlp_forward: NULL");
    if (M <= 0 || M % 128) return mfail(m, WX_EINVAL, "wx_mlp_forward: M must be a positive multiple of 128");
    cudaStream_t s = (cudaStream_t)stream;
    const __nv_bfloat16 *Xb = reinterpret_cast<const __nv_bfloat16 *>(X);
    // rows beyond the activation buffers go through in chunks of max_batch
    for (int r0 = 0; r0 < M; r0 += m->max_batch) {
        const int rows = std::min(m->max_batch, M - r0);
        const int rc = mlp_forward(m, Xb + (size_t)r0 * kXW, rows, Y + (size_t)r0 * kOutP, s, false);
        if (rc != WX_OK) return mfail(m, rc, m->err);
    }
    return WX_OK;
}

static int check_batch(wx_mlp *m, const void *X, const float *Yt, int M, const char *who) {
    if (!m) return WX_EINVAL;
    if (!X || !Yt) return mfail(m, WX_EINVAL, std::string(who) + ": NULL");
    if (M <= 0 || M % 128 || M > m->max_batch)
        return mfail(m, WX_EINVAL, std::string(who) + ": M must be a multiple of 128 and <= max_batch");
    return WX_OK;
}

extern "C" int wx_mlp_gradients(wx_mlp *m, const void *X, const float *Yt, int M, float *loss, void *stream) {
    int rc = check_batch(m, X, Yt, M, "wx_mlp_gradients");
    if (rc != WX_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const __nv_bfloat16 *Xb = reinterpret_cast<const __nv_bfloat16 *>(X);
    rc = mlp_forward(m, Xb, M, nullptr, s);
    if (rc == WX_OK) rc = mlp_backward(m, Xb, Yt, M, loss, s);
    if (rc != WX_OK) return mfail(m, rc, m->err);
    MCK(cudaGetLastError(), "gradient kernels");
    return WX_OK;
}

// One training step: forward, loss gradient, backward, then Adam with bias
// correction (beta1 0.9, beta2 0.999, eps 1e-8) on every weight and bias.
extern "C" int wx_mlp_train_step(wx_mlp *m, const void *X, const float *Yt, int M, float lr, float *loss,
                                 void *stream) {
    int rc = wx_mlp_gradients(m, X, Yt, M, loss, stream);
    if (rc != WX_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    ++m->adam_t;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)m->adam_t), c2 = 1.f - powf(b2, (float)m->adam_t);
    for (int l = 0; l < kLayers; ++l) {
        const int N = layer_out(l), K = layer_in(l);
        adam_kernel<<<grid1((long)N * K), 256, 0, s>>>(m->W[l], m->dW[l], m->mW[l], m->vW[l], (long)N * K, N, K, lr,
                                                      b1, b2, eps, c1, c2, l == 0, m->Wb[l],
                                                      l == 0 ? nullptr : m->WbT[l]);
        adam_kernel<<<grid1(N), 256, 0, s>>>(m->b[l], m->db[l], m->mb[l], m->vb[l], N, N, 1, lr, b1, b2, eps, c1,
                                            c2, 0, nullptr, nullptr);
    }
    MCK(cudaGetLastError(), "Adam kernels");
    return WX_OK;
}

extern "C" int wx_mlp_status(wx_mlp *m) {
    if (!m) return WX_EINVAL;
    unsigned st = 0;
    MCK(cudaMemcpy(&st, m->status, sizeof st, cudaMemcpyDeviceToHost), "status");
    if (st) cudaMemset(m->status, 0, sizeof st);
    if (st & ST_TIMEOUT) return mfail(m, WX_ETIMEOUT, "a bounded device wait timed out in a GEMM");
    return WX_OK;
}

// =====================================================================
// WX_SURROGATE: one time step with the column physics predicted by the
// network.  The dynamics kernel runs without physics and leaves T*, q* in
// the new buffer; the features of every column go through the four GEMMs;
// the apply kernel accepts a column's prediction only when both residual
// checks pass and otherwise recomputes the column exactly.
// =====================================================================
namespace wx {

constexpr int kSB = 64;          // columns per block of the feature and apply kernels
constexpr int kCS = 2 * kNZ;     // T* and q* values per column
constexpr int kCH = kInP / 8;    // 8-feature chunks per input row (32)
constexpr int kSC = (kCS + 7) / 8;  // chunks holding staged T*, q* (15)
constexpr int kFS = 8 * kSC + 1;    // staged row stride (odd)

// Normalised feature rows [rows][512] ([hi | lo], see kXW) of all nx*ny
// columns (raster order j*nx + i), straight from the planar T*, q* planes.
// Staging: thread t serves column t % kSB and every (threads / kSB)-th
// plane, its column's address computed once and all its loads issued back
// to back; value f of a column lands at (f % 8) kSC + f / 8 of its row, so
// that in the second phase -- one thread per (row, 8-feature chunk), a
// warp covering one row and writing its 512 contiguous bytes -- lanes read
// consecutive words.  Per-feature constants use the same [f % 8][f / 8]
// order; the inputs past T*, q* are s fa_f + fb_f (s = kappa_mult).
constexpr int kFeatThreads = 256;
__global__ void __launch_bounds__(kFeatThreads) sur_features_kernel(const float *__restrict__ fld, int nx, int P,
                                                                    int R, const float *__restrict__ km,
                                                                    const float *__restrict__ lev,
                                                                    const float *__restrict__ norm,
                                                                    __nv_bfloat16 *__restrict__ X, long ncol,
                                                                    long rows, long c0) {
    __shared__ float tile[kSB * kFS];
    __shared__ float smean[kInP], sinv[kInP], sfa[kInP], sfb[kInP], skm[kSB];
    const long r0 = (long)blockIdx.x * kSB;
    for (int f = threadIdx.x; f < kInP; f += blockDim.x) {
        const int d = (f % 8) * kCH + f / 8;
        smean[d] = f < kIn ? norm[f] : 0.f;
        sinv[d] = f < kIn ? 1.f / norm[kInP + f] : 0.f;
        sfa[d] = (f >= kCS && f < 3 * kNZ) ? lev[f - kCS] : 0.f;
        sfb[d] = (f >= 3 * kNZ && f < kIn) ? lev[kNZ + f - 3 * kNZ] : 0.f;
    }
    for (int e = threadIdx.x; e < kSB; e += blockDim.x) skm[e] = (km && r0 + e < ncol) ? km[c0 + r0 + e] : 1.f;
    {
        constexpr int G = kFeatThreads / kSB, PER = kCS / G;
        static_assert(kFeatThreads % kSB == 0 && kCS % G == 0, "plane split");
        const int u = threadIdx.x % kSB, g = threadIdx.x / kSB;
        const long c = r0 + u, cg = c0 + c;  // row of X, column of the grid
        const size_t plane = (size_t)R * P;
        float v[PER];
        if (c < ncol) {
            const int j = (int)(cg / nx), i = (int)(cg - (long)j * nx);
            const float *src = fld + (size_t)(j + 1) * P + i + kGhostX;
#pragma unroll
            for (int n = 0; n < PER; ++n) v[n] = src[(size_t)(g + n * G) * plane];
        } else {
#pragma unroll
            for (int n = 0; n < PER; ++n) v[n] = 0.f;
        }
#pragma unroll
        for (int n = 0; n < PER; ++n) {
            const int p = g + n * G, f = (p & 1) * kNZ + (p >> 1);  // plane (k, field) -> feature
            tile[u * kFS + (f % 8) * kSC + f / 8] = v[n];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kSB * kCH; e += blockDim.x) {
        const int r = e / kCH, g = e % kCH;
        const long row = r0 + r;
        if (row >= rows) continue;
        const float live = row < ncol ? 1.f : 0.f;
        const float s = skm[r];
        __align__(16) __nv_bfloat162 hi[4], lo[4];
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
            float x[2];
#pragma unroll
            for (int w = 0; w < 2; ++w) {
                const int d = (u + w) * kCH + g;
                const float staged = 8 * g + u + w < kCS ? tile[r * kFS + (u + w) * kSC + g] : 0.f;
                const float raw = staged + s * sfa[d] + sfb[d];
                x[w] = live * ((raw - smean[d]) * sinv[d]);
            }
            const __nv_bfloat162 h = __floats2bfloat162_rn(x[0], x[1]);
            hi[u / 2] = h;
            lo[u / 2] = __floats2bfloat162_rn(x[0] - __low2float(h), x[1] - __high2float(h));
        }
        __nv_bfloat16 *dst = X + row * kXW + 8 * g;
        *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(hi);
        *reinterpret_cast<uint4 *>(dst + kInP) = *reinterpret_cast<const uint4 *>(lo);
    }
}

// Columns of a block of kSB consecutive raster columns staged in shared
// memory for the apply kernel, row-major [column][CS] = [T*_0..57 | q*_0..57 | pad], by
// coalesced plane reads: thread t serves column t % kSB and every
// (NTH / kSB)-th plane, its column's address computed once, all its loads
// issued back to back (an unrolled loop with no dependence between them).
template <int NTH, int CS>
__device__ __forceinline__ void stage_columns(float *tile, const float *__restrict__ fld, long r0, long ncol,
                                              int nx, int P, size_t plane) {
    static_assert(NTH % kSB == 0 && kCS % (NTH / kSB) == 0, "plane split");
    constexpr int G = NTH / kSB, PER = kCS / G;
    const int u = threadIdx.x % kSB, g = threadIdx.x / kSB;
    const long c = r0 + u;
    if (c < ncol) {
        const int j = (int)(c / nx), i = (int)(c - (long)j * nx);
        const float *src = fld + (size_t)(j + 1) * P + i + kGhostX;
        float v[PER];
#pragma unroll
        for (int n = 0; n < PER; ++n) v[n] = src[(size_t)(g + n * G) * plane];
#pragma unroll
        for (int n = 0; n < PER; ++n) {
            const int p = g + n * G;                 // plane (k, f), f = p & 1
            tile[u * CS + (p & 1) * kNZ + (p >> 1)] = v[n];
        }
    } else {
#pragma unroll 4
        for (int n = 0; n < PER; ++n) {
            const int p = g + n * G;
            tile[u * CS + (p & 1) * kNZ + (p >> 1)] = 0.f;
        }
    }
}

// Residual checks, fallback and T^{n+1} for a block of kSB columns: the
// columns' T*, q* and their output rows are staged in shared memory; one
// thread per column then runs the checks (and, for a rejected column, the
// exact elimination, back substitution and scan) on shared data only, and
// writes its new T column back with the periodic ghost copies (a warp's
// stores to one plane are coalesced).  Row strides are odd, so a thread
// walking its own row hits distinct banks.  Two threads per column share
// the loads and stores; the first kSB threads do the per-column work.
constexpr int kYS = kOut + 1;   // row stride of the staged outputs
constexpr int kTS = kCS + 1;    // row stride of the staged columns
constexpr int kApplyThreads = 2 * kSB;
__global__ void __launch_bounds__(kApplyThreads) sur_apply_kernel(float *__restrict__ fld, int nx, int ny, int P, int R,
                                                        const float *__restrict__ km,
                                                        const Q4<float> *__restrict__ gtab,
                                                        const float *__restrict__ Y,
                                                        const float *__restrict__ norm, float dt, float S0,
                                                        float tol, long ncol,
                                                        unsigned long long *__restrict__ n_fallback,
                                                        unsigned *__restrict__ status, long c0,
                                                        int count_only) {
    extern __shared__ __align__(16) float dsm[];
    float *tile = dsm;                  // [kSB][kTS] T* | q*; T* is overwritten by T^{n+1}
    float *ysm = dsm + kSB * kTS;       // [kSB][kYS] outputs, then scratch
    __shared__ Q4<float> sB[kNZ], sC[kNZ], sE[kNZ];
    __shared__ float smo[kOut], sso[kOut];
    const int t = threadIdx.x;
    const long r0 = (long)blockIdx.x * kSB;
    const size_t plane = (size_t)R * P;
    for (int e = t; e < kNZ; e += blockDim.x) {
        sB[e] = gtab[REC_B * kNZ + e];
        sC[e] = gtab[REC_C * kNZ + e];
        sE[e] = gtab[REC_E * kNZ + e];
    }
    for (int e = t; e < kOut; e += blockDim.x) {
        smo[e] = norm[2 * kInP + e];
        sso[e] = norm[3 * kInP + e];
    }
    {   // output rows: warp w reads rows 16 w .. 16 w + 15, one 464-byte row
        // (29 lanes x 16 bytes) per load, all 16 loads in flight
        constexpr int RPW = kSB / (kApplyThreads / 32);
        const int w = t / 32, lane = t % 32;
        float4 buf[RPW];
#pragma unroll
        for (int n = 0; n < RPW; ++n) {
            const long row = r0 + w * RPW + n;
            buf[n] = (lane < kOut / 4 && row < ncol)
                         ? reinterpret_cast<const float4 *>(Y + row * kOutP)[lane]
                         : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int n = 0; n < RPW; ++n) {
            if (lane < kOut / 4) {
                float *d = ysm + (w * RPW + n) * kYS + 4 * lane;
                d[0] = buf[n].x;
                d[1] = buf[n].y;
                d[2] = buf[n].z;
                d[3] = buf[n].w;
            }
        }
    }
    stage_columns<kApplyThreads, kTS>(tile, fld, c0 + r0, c0 + ncol, nx, P, plane);
    __syncthreads();
    const long c = r0 + t;
    bool reject = false, ok = true;
    if (t < kSB && c < ncol) {
        float *yr = ysm + t * kYS;
        float *ts = tile + t * kTS, *qs = ts + kNZ;
        for (int o = 0; o < kOut; ++o) yr[o] = fmaf(yr[o], sso[o], smo[o]);  // H_k | r_k
        const float s = km ? km[c0 + c] : 1.f;
        // rho_vd: (A v - T*)_k = (v_k - T*_k) + a_k (v_{k-1} - v_k) + c_k (v_{k+1} - v_k)
        // with v = T* + dt r; level differences of T* first (exact in FP32
        // for neighbouring values) so that dt r never rounds against T ~ 300
        float num = 0.f, den = 0.f, sumH = 0.f, tau2 = 0.f;
        bool finite = true;
#pragma unroll 2
        for (int k = 0; k < kNZ; ++k) {
            const float ak = s * sE[k].x, ck = s * sE[k].y;
            const float tk = ts[k], rk = yr[kNZ + k];
            const float dtm = k > 0 ? ts[k - 1] - tk : 0.f, dtp = k < kNZ - 1 ? ts[k + 1] - tk : 0.f;
            const float drm = k > 0 ? yr[kNZ + k - 1] - rk : 0.f, drp = k < kNZ - 1 ? yr[kNZ + k + 1] - rk : 0.f;
            const float e0 = ak * dtm + ck * dtp;
            const float ex = e0 + dt * (rk + ak * drm + ck * drp);
            num = fmaf(ex, ex, num);
            den = fmaf(e0, e0, den);
            sumH = fmaf(yr[k], sE[k].z, sumH);
            tau2 = fmaf(sB[k].z, qs[k], tau2);
            finite = finite && isfinite(yr[k]) && isfinite(rk);
        }
        const float absorbed = S0 * (1.f - exp2f(-tau2));
        const float rvd = den > 0.f ? sqrtf(num / den) : (num == 0.f ? 0.f : INFINITY);
        const float rH = absorbed > 0.f ? fabsf(sumH - absorbed) / absorbed : (sumH == 0.f ? 0.f : INFINITY);
        reject = !(finite && rvd <= tol && rH <= tol);
        if (count_only) {
            // acceptance probe: the verdict alone
        } else if (!reject) {
            for (int k = 0; k < kNZ; ++k) ts[k] = ts[k] + dt * (yr[kNZ + k] + yr[k]);
        } else {
            // exact column: forward elimination (c'_k, d'_k in the row's
            // scratch), back substitution with the heating of the
            // optical-depth scan from the top
            float *cp = yr, *dp = yr + kNZ;
            ThomasSweep<float> fw;
            for (int k = 0; k < kNZ; ++k) {
                cp[k] = fw.level(-s * sE[k].x, -s * sE[k].y, ts[k]);
                dp[k] = fw.d;
            }
            float x = 0.f, tau = 0.f, Etop = 1.f;
            for (int k = kNZ - 1; k >= 0; --k) {
                x = dp[k] - cp[k] * x;
                const float taub = tau + sB[k].z * qs[k];
                const float Eb = exp2f(-taub);
                ts[k] = x + sC[k].x * (Etop - Eb);
                Etop = Eb;
                tau = taub;
            }
        }
        for (int k = 0; k < kNZ; ++k) ok = ok && isfinite(ts[k]);
    }
    const int nrej = __syncthreads_count(reject);
    if (!__syncthreads_and(ok) && t == 0) atomicOr(status, ST_NONFINITE);
    if (t == 0 && nrej) atomicAdd(n_fallback, (unsigned long long)nrej);
    if (count_only) return;
    const int u = t % kSB, half = t / kSB;
    const long cu = r0 + u;
    if (cu < ncol) {
        const long cg = c0 + cu;
        const int j = (int)(cg / nx), i = (int)(cg - (long)j * nx);
        float *col = fld + (size_t)(j + 1) * P + i + kGhostX;
        const float *ts = tile + u * kTS;
#pragma unroll 4
        for (int k = half; k < kNZ; k += kApplyThreads / kSB) {
            const float v = ts[k];
            float *row = col + (size_t)(2 * k) * plane;
            row[0] = v;
            if (i == 0) row[nx] = v;                   // -> right ghost column
            if (i == nx - 1) row[-nx] = v;             // -> left ghost column
            if (j == 0) row[(size_t)ny * P] = v;       // -> top ghost row
            if (j == ny - 1) row[-(long)ny * P] = v;   // -> bottom ghost row
        }
    }
}

static void free_policy(wx_ctx *c);

void free_surrogate(wx_ctx *c) {
    free_policy(c);
    for (void *p : {c->sur_X, c->sur_H[0], c->sur_H[1], (void *)c->sur_Y, (void *)c->sur_lev, (void *)c->sur_nfb})
        if (p) cudaFree(p);
    c->sur_X = c->sur_H[0] = c->sur_H[1] = nullptr;
    c->sur_Y = c->sur_lev = nullptr;
    c->sur_nfb = nullptr;
    c->sur = nullptr;
    c->sur_rows = 0;
}

// The network on the raster columns [c0, c0 + ncol) of state buffer f,
// which holds T* and q* there: features, the four GEMMs, the residual
// checks.  count_only counts the rejected columns into *counter and writes
// nothing; otherwise accepted predictions and exact fallbacks become
// T^{n+1} and *counter counts the fallbacks.
static int run_network(wx_ctx *c, float *f, long c0, long ncol, bool count_only, unsigned long long *counter,
                       cudaStream_t s, long *launches) {
    wx_mlp *m = c->sur;
    const long rows = (ncol + 127) / 128 * 128;
    cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    sur_features_kernel<<<(unsigned)((rows + kSB - 1) / kSB), kFeatThreads, 0, s>>>(
        f, c->nx, c->P, c->R, (const float *)c->kmult, c->sur_lev, m->norm,
        reinterpret_cast<__nv_bfloat16 *>(c->sur_X), ncol, rows, c0);
    std::string err;
    const int M = (int)rows;
    const __nv_bfloat16 *X = reinterpret_cast<const __nv_bfloat16 *>(c->sur_X);
    __nv_bfloat16 *H0 = reinterpret_cast<__nv_bfloat16 *>(c->sur_H[0]);
    __nv_bfloat16 *H1 = reinterpret_cast<__nv_bfloat16 *>(c->sur_H[1]);
    int rc = gemm(X, m->Wb[0], M, kHid, kXW, EPI_GELU, m->b[0], nullptr, H0, nullptr, c->d_status, s, err);
    if (rc == WX_OK) rc = gemm(H0, m->Wb[1], M, kHid, kHid, EPI_GELU, m->b[1], nullptr, H1, nullptr, c->d_status, s, err);
    if (rc == WX_OK) rc = gemm(H1, m->Wb[2], M, kHid, kHid, EPI_GELU, m->b[2], nullptr, H0, nullptr, c->d_status, s, err);
    if (rc == WX_OK)
        rc = gemm(H0, m->Wb[3], M, kOutP, kHid, EPI_F32, m->b[3], nullptr, c->sur_Y, nullptr, c->d_status, s, err);
    if (rc != WX_OK) {
        c->err = err;
        return rc;
    }
    constexpr int apply_smem = kSB * (kTS + kYS) * (int)sizeof(float);
    {   // a per-device function attribute: set on every launch (cheap)
        cudaError_t e = cudaFuncSetAttribute(sur_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, apply_smem);
        if (e != cudaSuccess) {
            c->err = std::string("surrogate apply attribute: ") + cudaGetErrorString(e);
            return WX_ECUDA;
        }
    }
    sur_apply_kernel<<<(unsigned)((ncol + kSB - 1) / kSB), kApplyThreads, apply_smem, s>>>(
        f, c->nx, c->ny, c->P, c->R, (const float *)c->kmult, (const Q4<float> *)c->tab, c->sur_Y, m->norm,
        (float)c->dt, (float)c->S0, (float)c->sur_tol, ncol, counter, c->d_status, c0, count_only ? 1 : 0);
    *launches += 6;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        c->err = std::string("surrogate kernels: ") + cudaGetErrorString(e);
        return WX_ECUDA;
    }
    return WX_OK;
}

static int surrogate_levels(wx_ctx *c) {
    if (c->sur_gen == c->generation) return WX_OK;
    // per-level feature inputs from this context's parameters
    std::vector<float> lev(2 * kNZ);
    for (int k = 0; k < kNZ; ++k) {
        lev[k] = (float)c->kappa_lev[k];
        lev[kNZ + k] = (float)(c->alpha[k] * c->dz[k]);
    }
    cudaError_t e = cudaMemcpy(c->sur_lev, lev.data(), lev.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        c->err = std::string("surrogate levels: ") + cudaGetErrorString(e);
        return WX_ECUDA;
    }
    c->sur_gen = c->generation;
    return WX_OK;
}

int launch_surrogate_step(wx_ctx *c, cudaStream_t s, long *launches) {
    int rc = surrogate_levels(c);
    if (rc != WX_OK) return rc;
    // 1. dynamics only: T*, q* land in the new buffer (which becomes current)
    const unsigned saved = c->flags;
    c->flags = saved & WX_ADVECTION;
    rc = launch_step(c, s, launches);
    c->flags = saved;
    if (rc != WX_OK) return rc;
    // 2. features, the network, residual checks, fallback, T^{n+1}
    return run_network(c, reinterpret_cast<float *>(c->fld[c->cur]), 0, (long)c->nx * c->ny, false, c->sur_nfb, s,
                       launches);
}

// ------------------------------------------------- the acceptance policy
void reset_surrogate_policy(wx_ctx *c) {
    for (const auto &r : c->sur_reads) cudaEventSynchronize(c->sur_ev[r.slot]);
    c->sur_reads.clear();
    c->sur_mode = 0;
    c->sur_last_exact = false;
    c->sur_step = c->sur_next_probe = 0;
    c->sur_probe_row0 = 0;
}

static void free_policy(wx_ctx *c) {
    reset_surrogate_policy(c);
    for (auto &ev : c->sur_ev)
        if (ev) {
            cudaEventDestroy(ev);
            ev = nullptr;
        }
    if (c->sur_host) cudaFreeHost(c->sur_host);
    c->sur_host = nullptr;
}

// The counts of the steps up to `upto` decide the mode: network steps while
// the acceptance is at least the policy's minimum, exact steps otherwise.
static int resolve_reads(wx_ctx *c, long long upto, long long now) {
    while (!c->sur_reads.empty() && c->sur_reads.front().step <= upto) {
        const wx_ctx::SurRead r = c->sur_reads.front();
        c->sur_reads.erase(c->sur_reads.begin());
        if (cudaEventSynchronize(c->sur_ev[r.slot]) != cudaSuccess) {
            c->err = "surrogate policy: reading an acceptance count failed";
            return WX_ECUDA;
        }
        const double accept = 1.0 - (double)c->sur_host[r.slot] / (double)r.ncols;
        if (accept >= c->sur_min_accept) {
            c->sur_mode = 0;
        } else if (c->sur_mode == 0) {
            c->sur_mode = 1;
            c->sur_next_probe = now + c->sur_probe_every;
        }
    }
    return WX_OK;
}

static int record_count(wx_ctx *c, long long step, long ncols, const unsigned long long *counter, cudaStream_t s) {
    if ((int)c->sur_reads.size() >= wx_ctx::kSurRing) {
        const int rc = resolve_reads(c, c->sur_reads.front().step, step);
        if (rc != WX_OK) return rc;
    }
    const int slot = c->sur_slot;
    c->sur_slot = (slot + 1) % wx_ctx::kSurRing;
    if (cudaMemcpyAsync(&c->sur_host[slot], counter, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaEventRecord(c->sur_ev[slot], s) != cudaSuccess) {
        c->err = "surrogate policy: enqueueing an acceptance count failed";
        return WX_ECUDA;
    }
    c->sur_reads.push_back({step, ncols, slot});
    return WX_OK;
}

int launch_surrogate_policy_step(wx_ctx *c, cudaStream_t s, long *launches) {
    if (c->sur_min_accept <= 0.0) {  // no policy: the network runs every step
        c->sur_last_exact = false;
        return launch_surrogate_step(c, s, launches);
    }
    if (!c->sur_host) {
        bool ok = cudaHostAlloc((void **)&c->sur_host, wx_ctx::kSurRing * sizeof(unsigned long long),
                                cudaHostAllocDefault) == cudaSuccess;
        for (auto &ev : c->sur_ev) ok = ok && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            free_policy(c);
            c->err = "surrogate policy: pinned count buffer or events unavailable";
            return WX_ENOMEM;
        }
    }
    const long long n = c->sur_step;
    int rc = resolve_reads(c, n - 2, n);
    if (rc != WX_OK) return rc;
    c->sur_step = n + 1;
    if (c->sur_mode == 0) {
        c->sur_last_exact = false;
        rc = launch_surrogate_step(c, s, launches);
        return rc == WX_OK ? record_count(c, n, (long)c->nx * c->ny, c->sur_nfb, s) : rc;
    }
    // exact step: the fused kernel with the column physics
    c->sur_last_exact = true;
    rc = launch_step(c, s, launches);
    if (rc != WX_OK || n < c->sur_next_probe) return rc;
    // probe: the network on a band of rows of the new state, verdicts only
    rc = surrogate_levels(c);
    if (rc != WX_OK) return rc;
    const int rows = std::min(c->sur_probe_rows, c->ny);
    int j0 = c->sur_probe_row0;
    if (j0 + rows > c->ny) j0 = 0;
    c->sur_probe_row0 = (j0 + rows) % c->ny;
    c->sur_next_probe = n + c->sur_probe_every;
    const long ncol = (long)rows * c->nx;
    rc = run_network(c, reinterpret_cast<float *>(c->fld[c->cur]), (long)j0 * c->nx, ncol, true, c->sur_nfb + 1, s,
                     launches);
    return rc == WX_OK ? record_count(c, n, ncol, c->sur_nfb + 1, s) : rc;
}

}  // namespace wx

extern "C" int wx_set_surrogate(wx_ctx *c, wx_mlp *m, double fallback_tol) {
    if (!c) return WX_EINVAL;
    if (!m) {
        free_surrogate(c);
        return WX_OK;
    }
    if (c->dtype != WX_F32 || c->nz != kNZ) {
        c->err = "wx_set_surrogate: the network serves FP32 contexts with 58 levels";
        return WX_EUNSUPPORTED;
    }
    if (!(fallback_tol >= 0) || !std::isfinite(fallback_tol)) {
        c->err = "wx_set_surrogate: fallback_tol must be finite and >= 0";
        return WX_EINVAL;
    }
    free_surrogate(c);
    const long rows = ((long)c->nx * c->ny + 127) / 128 * 128;
    bool ok = cudaMalloc(&c->sur_X, rows * kXW * 2) == cudaSuccess &&
              cudaMalloc(&c->sur_H[0], rows * kHid * 2) == cudaSuccess &&
              cudaMalloc(&c->sur_H[1], rows * kHid * 2) == cudaSuccess &&
              cudaMalloc((void **)&c->sur_Y, rows * kOutP * 4) == cudaSuccess &&
              cudaMalloc((void **)&c->sur_lev, 2 * kNZ * 4) == cudaSuccess &&
              cudaMalloc((void **)&c->sur_nfb, 2 * sizeof(unsigned long long)) == cudaSuccess &&
              cudaMemset(c->sur_nfb, 0, 2 * sizeof(unsigned long long)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_surrogate(c);
        c->err = "wx_set_surrogate: device allocation failed";
        return WX_ENOMEM;
    }
    c->sur = m;
    c->sur_rows = rows;
    c->sur_tol = fallback_tol;
    c->sur_gen = ~0u;
    return WX_OK;
}

extern "C" int wx_surrogate_fallbacks(wx_ctx *c, long *n_fallback) {
    if (!c || !n_fallback) return WX_EINVAL;
    if (!c->sur_nfb) {
        c->err = "wx_surrogate_fallbacks: no network attached";
        return WX_ESTATE;
    }
    unsigned long long n = 0;
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(&n, c->sur_nfb, sizeof n, cudaMemcpyDeviceToHost) != cudaSuccess) {
        c->err = "wx_surrogate_fallbacks: device error";
        return WX_ECUDA;
    }
    // an exact step (the policy skipped the network) computed every column exactly
    *n_fallback = c->sur_last_exact ? (long)c->nx * c->ny : (long)n;
    return WX_OK;
}

extern "C" int wx_set_surrogate_policy(wx_ctx *c, double min_accept, int probe_every, int probe_rows) {
    if (!c) return WX_EINVAL;
    if (!(min_accept >= 0.0 && min_accept <= 1.0) || probe_every < 1 || probe_rows < 1) {
        c->err = "wx_set_surrogate_policy: min_accept in [0, 1], probe_every >= 1, probe_rows >= 1";
        return WX_EINVAL;
    }
    reset_surrogate_policy(c);
    c->sur_min_accept = min_accept;
    c->sur_probe_every = probe_every;
    c->sur_probe_rows = probe_rows;
    return WX_OK;
}
