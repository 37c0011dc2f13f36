// wx_step.cu -- the fused weather-step kernel and its helpers.
//
// One CTA owns a 32 x TY tile of columns and walks it bottom to top once
// (pass 1) and top to bottom once (pass 2):
//
//   pass 1, level k = 0 .. nz-1
//     TMA stages k-slabs of the (T, q) cell array, tile plus a one-cell halo,
//     into a ring of shared-memory stages (mbarrier completion).  Each thread
//     forms phi* for its column at level k from the 5-point horizontal
//     neighbourhood in shared memory and the vertical neighbours it carries in
//     registers (dynamics, paper Eq. 1 + upwind advection), then runs the
//     Thomas forward elimination of the implicit vertical diffusion for T*
//     (the K dependency the paper keeps sequential, Sec. 2.2) and parks c'_k,
//     d'_k and q*_k in shared memory.
//   pass 2, level k = nz-1 .. 0
//     back substitution x_k = d'_k - c'_k x_{k+1}, the optical-depth scan from
//     the top and the heating H_k, then one 8-byte (16-byte in FP64) store of
//     the new (T, q) cell, plus ghost-ring copies from edge tiles.
//
// Each field crosses HBM once per step in each direction.  The horizontal
// operator is rewritten as per-column coefficients
//   phi* = cC phi + cE phi_E + cW phi_W + cN phi_N + cS phi_S
//          + wU_k (phi_{k+1} - phi_k) - wD_k (phi_k - phi_{k-1}),
// with the upwind choice folded into cE..cS (U+ = max(U,0), U- = min(U,0)):
//   cE = dh - dth Ue-,  cW = dh + dth Uw+,  cN = dh - dth Vn-,  cS = dh + dth Vs+,
//   cC = 1 - 4 dh - dth (Ue+ - Uw- + Vn+ - Vs-),
// the same linear map as the flux form, evaluated in a different order.
#include <cstdio>

#include "ptx.cuh"
#include "wx_internal.cuh"

namespace wx {

template <typename T> __device__ __forceinline__ T exp_neg(T x);
template <> __device__ __forceinline__ float exp_neg<float>(float x) { return __expf(-x); }
template <> __device__ __forceinline__ double exp_neg<double>(double x) { return exp(-x); }

template <typename T> __device__ __forceinline__ T recip(T m);
template <> __device__ __forceinline__ float recip<float>(float m) { return __frcp_rn(m); }
template <> __device__ __forceinline__ double recip<double>(double m) { return 1.0 / m; }

template <typename T> __device__ __forceinline__ bool finite(T x) { return isfinite(x); }

// Column sum of phi*dz in the storage precision, compensated in FP32 so the
// FP64 total that follows is not limited by a 58-term FP32 sum.
template <typename T> struct ColSum;
template <> struct ColSum<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v, float w) {
        const float p = v * w;
        const float pe = fmaf(v, w, -p);  // exact product error
        const float s1 = s + p;           // TwoSum(s, p)
        const float bp = s1 - s;
        const float e = (s - (s1 - bp)) + (p - bp);
        c += e + pe;
        s = s1;
    }
    __device__ __forceinline__ double total() const { return (double)s + (double)c; }
};
template <> struct ColSum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double v, double w) { s = fma(v, w, s); }
    __device__ __forceinline__ double total() const { return s; }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

template <typename T, int TY, int KB, bool PHYS, bool SUMS>
__global__ void __launch_bounds__(32 * TY) step_kernel(const __grid_constant__ CUtensorMap tin,
                                                       const StepArgs<T> a, const int S) {
    using C2 = typename Vec2<T>::type;
    constexpr int NT = 32 * TY;
    constexpr int PC = (TY + 2) * kBoxX;  // cells per staged plane
    extern __shared__ __align__(128) unsigned char smem[];

    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + 32 * ty;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int i = blockIdx.x * kTileX + tx, j = blockIdx.y * TY + ty;
    const bool valid = (i < nx) && (j < ny);

    const SmemPlan pl = plan_smem(nz, TY, S, KB, (int)sizeof(C2), (int)sizeof(T), PHYS ? 3 : 2);
    T *tab = reinterpret_cast<T *>(smem + pl.tab_off);
    C2 *ring = reinterpret_cast<C2 *>(smem + pl.ring_off);
    T *st_dp = reinterpret_cast<T *>(smem + pl.state_off);
    T *st_qs = st_dp + nz * NT;
    T *st_cp = st_qs + nz * NT;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + pl.bar_off);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(full + S);

    const int n_stages = (nz + KB - 1) / KB;
    const int SC = pl.stage_bytes / (int)sizeof(C2);  // cells per stage slot
    constexpr int wpc = (int)(sizeof(C2) / 4);  // 32-bit words per cell
    const int x0 = (kGhostX - 2 + (int)blockIdx.x * kTileX) * wpc;
    const int y0 = (int)blockIdx.y * TY;
    const uint32_t stage_tx = (uint32_t)(KB * PC * sizeof(C2));

    if (tid == 0) {
        prefetch_tmap(&tin);
        for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
        *abort_flag = 0;
        fence_mbar_init();
        const int first = n_stages < S ? n_stages : S;
        for (int s = 0; s < first; ++s) {
            mbar_arrive_expect_tx(&full[s], stage_tx);
            tma_load_3d(ring + s * SC, &tin, &full[s], x0, y0, s * KB);
        }
    }
    for (int e = tid; e < nz * kTab; e += NT) tab[e] = a.tab[e];

    // per-column coefficients of the horizontal operator
    const int ic = valid ? i : 0, jc = valid ? j : 0;
    T ue = 0, uw = 0, vn = 0, vs = 0;
    if (a.advection) {
        ue = a.U[(size_t)jc * nx + ic];
        uw = a.U[(size_t)jc * nx + (ic == 0 ? nx - 1 : ic - 1)];
        vn = a.V[(size_t)jc * nx + ic];
        vs = a.V[(size_t)(jc == 0 ? ny - 1 : jc - 1) * nx + ic];
    }
    const T zero = T(0);
    const T cE = a.dh - a.dth * fmin(ue, zero);
    const T cW = a.dh + a.dth * fmax(uw, zero);
    const T cN = a.dh - a.dth * fmin(vn, zero);
    const T cS = a.dh + a.dth * fmax(vs, zero);
    const T cC = T(1) - T(4) * a.dh -
                 a.dth * (fmax(ue, zero) - fmin(uw, zero) + fmax(vn, zero) - fmin(vs, zero));
    const T km = a.kmult ? a.kmult[(size_t)jc * nx + ic] : T(1);

    __syncthreads();  // barriers initialised, table staged

    bool ok = mbar_wait_bounded(&full[0], 0);
    const int ctr = (ty + 1) * kBoxX + tx + 2;
    C2 cur = ring[ctr];
    C2 prev = cur;
    T cp_prev = 0, dp_prev = 0;

    // plane k lives in stage k/KB, slot (k/KB) % S, sub-plane k % KB
    int sub = 0, slot = 0, gst = 0;       // plane k
    int sub1 = 1 % KB, slot1 = (KB == 1) ? 1 % S : 0;
    uint32_t par1 = (KB == 1 && S == 1) ? 1u : 0u;
    for (int k = 0; k < nz; ++k) {
        const C2 *pk = ring + slot * SC + sub * PC;
        C2 nxt = cur;
        if (k + 1 < nz) {
            if (sub1 == 0) ok &= mbar_wait_bounded(&full[slot1], par1);
            nxt = ring[slot1 * SC + sub1 * PC + ctr];
        }
        const C2 e = pk[ctr + 1], w = pk[ctr - 1], n = pk[ctr + kBoxX], s = pk[ctr - kBoxX];
        const T wU = tab[k * kTab + TAB_WU], wD = tab[k * kTab + TAB_WD];

        const T ts = cC * cur.x + cE * e.x + cW * w.x + cN * n.x + cS * s.x + wU * (nxt.x - cur.x) -
                     wD * (cur.x - prev.x);
        const T qs = cC * cur.y + cE * e.y + cW * w.y + cN * n.y + cS * s.y + wU * (nxt.y - cur.y) -
                     wD * (cur.y - prev.y);
        if (PHYS) {
            const T ak = km * tab[k * kTab + TAB_AHAT];
            const T ck = km * tab[k * kTab + TAB_CHAT];
            const T bk = T(1) - ak - ck;
            const T m = bk - ak * cp_prev;
            const T inv = recip(m);
            const T cp = ck * inv;
            const T dp = (ts - ak * dp_prev) * inv;
            st_cp[k * NT + tid] = cp;
            st_dp[k * NT + tid] = dp;
            cp_prev = cp;
            dp_prev = dp;
        } else {
            st_dp[k * NT + tid] = ts;
        }
        st_qs[k * NT + tid] = qs;
        prev = cur;
        cur = nxt;

        // advance plane k+1 cursor
        if (++sub1 == KB) {
            sub1 = 0;
            if (++slot1 == S) { slot1 = 0; par1 ^= 1u; }
        }
        // plane k's stage done: refill its slot with stage gst + S
        if (++sub == KB) {
            sub = 0;
            if (!ok) *abort_flag = 1;
            __syncthreads();
            if (*abort_flag) {
                if (tid == 0) {
                    atomicOr(a.status, ST_TIMEOUT);
                    // bounded wait for the last fill of every slot, so no copy
                    // is still landing in shared memory when the CTA exits
                    const int issued = (gst + S < n_stages) ? gst + S : n_stages;
                    for (int s2 = 0; s2 < S && s2 < issued; ++s2) {
                        const int fills = (issued - 1 - s2) / S;
                        (void)mbar_wait_bounded(&full[s2], (uint32_t)(fills & 1));
                    }
                }
                return;
            }
            if (tid == 0 && (gst + S) < n_stages) {
                mbar_arrive_expect_tx(&full[slot], stage_tx);
                tma_load_3d(ring + slot * SC, &tin, &full[slot], x0, y0, (gst + S) * KB);
            }
            ++gst;
            if (++slot == S) slot = 0;
        }
    }
    if (!ok && tid == 0) atomicOr(a.status, ST_TIMEOUT);

    // pass 2: back substitution, radiation scan from the top, store
    const size_t plane = (size_t)a.R * a.P;
    const int ip = i + kGhostX, jp = j + 1;
    C2 *out = a.out;
    T x = 0, tau = 0, Etop = 1;
    T chk = 0;
    ColSum<T> sumT, sumQ;
    for (int k = nz - 1; k >= 0; --k) {
        const T dp = st_dp[k * NT + tid];
        const T qs = st_qs[k * NT + tid];
        T tn;
        if (PHYS) {
            x = dp - st_cp[k * NT + tid] * x;
            const T taub = tau + tab[k * kTab + TAB_WTAU] * qs;
            const T Eb = exp_neg(taub);
            tn = x + tab[k * kTab + TAB_WH] * (Etop - Eb);
            Etop = Eb;
            tau = taub;
        } else {
            tn = dp;
        }
        if (valid) {
            C2 v;
            v.x = tn;
            v.y = qs;
            C2 *row = out + (size_t)k * plane + (size_t)jp * a.P;
            row[ip] = v;
            if (i == 0) row[kGhostX + nx] = v;
            if (i == nx - 1) row[kGhostX - 1] = v;
            if (j == 0) out[(size_t)k * plane + (size_t)(ny + 1) * a.P + ip] = v;
            if (j == ny - 1) out[(size_t)k * plane + ip] = v;
            if (SUMS) {
                const T dzk = tab[k * kTab + TAB_DZ];
                sumT.add(tn, dzk);
                sumQ.add(qs, dzk);
            } else {
                chk += tn + qs;
            }
        }
    }

    double mT = 0.0, mQ = 0.0;
    if (valid) {
        if (SUMS) {
            mT = sumT.total();
            mQ = sumQ.total();
            if (!isfinite(mT) || !isfinite(mQ)) atomicOr(a.status, ST_NONFINITE);
        } else if (!finite(chk)) {
            atomicOr(a.status, ST_NONFINITE);
        }
    }
    if (SUMS) {
        // deterministic CTA reduction: warp tree, then warps in order
        mT = warp_sum(mT);
        mQ = warp_sum(mQ);
        __syncthreads();  // ring no longer read by anyone
        double *red = reinterpret_cast<double *>(ring);
        if (tx == 0) {
            red[2 * ty] = mQ;
            red[2 * ty + 1] = mT;
        }
        __syncthreads();
        if (tid == 0) {
            double q = 0.0, t = 0.0;
            for (int w = 0; w < TY; ++w) {
                q += red[2 * w];
                t += red[2 * w + 1];
            }
            const size_t b = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
            a.partials[2 * b] = q;
            a.partials[2 * b + 1] = t;
        }
    }
}

// Fixed-order FP64 reduction of the per-CTA partials into one ring entry.
__global__ void __launch_bounds__(1024) sums_finalize(const double *__restrict__ part, long nblk, double h2,
                                                      double *__restrict__ dst) {
    __shared__ double sq[1024], st[1024];
    double q = 0.0, t = 0.0;
    for (long b = threadIdx.x; b < nblk; b += blockDim.x) {
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
        dst[0] = h2 * sq[0];
        dst[1] = h2 * st[0];
    }
}

// Per-level tables from FP64 dz, kappa_lev, alpha (one thread per level).
template <typename T>
__global__ void tables_kernel(const double *lev, int nz, double dt, double kappa_h, double S0, double q_ref,
                              T *tab) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nz) return;
    const double *dz = lev, *kl = lev + nz, *al = lev + 2 * nz;
    double wU = 0, wD = 0, ah = 0, ch = 0;
    if (k < nz - 1) {
        const double g = 0.5 * (dz[k] + dz[k + 1]);
        wU = dt * kappa_h / (dz[k] * g);
        ch = -dt * (0.5 * (kl[k] + kl[k + 1])) / (dz[k] * g);
    }
    if (k > 0) {
        const double g = 0.5 * (dz[k - 1] + dz[k]);
        wD = dt * kappa_h / (dz[k] * g);
        ah = -dt * (0.5 * (kl[k - 1] + kl[k])) / (dz[k] * g);
    }
    T *r = tab + k * kTab;
    r[TAB_WU] = (T)wU;
    r[TAB_WD] = (T)wD;
    r[TAB_AHAT] = (T)ah;
    r[TAB_CHAT] = (T)ch;
    r[TAB_WTAU] = (T)(al[k] * dz[k] / q_ref);
    r[TAB_WH] = (T)(dt * S0 / dz[k]);
    r[TAB_DZ] = (T)dz[k];
    r[TAB_PAD] = (T)0;
}

// FP64 [nz][ny][nx] (T, q) -> padded interleaved cells with the ghost ring.
template <typename T>
__global__ void pack_kernel(const double *__restrict__ Tsrc, const double *__restrict__ qsrc,
                            typename Vec2<T>::type *__restrict__ dst, int nx, int ny, int nz, int P, int R) {
    using C2 = typename Vec2<T>::type;
    const size_t n = (size_t)P * R * nz;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int ip = (int)(e % P);
        const int jp = (int)((e / P) % R);
        const int k = (int)(e / ((size_t)P * R));
        C2 v;
        v.x = 0;
        v.y = 0;
        if (ip >= kGhostX - 1 && ip <= kGhostX + nx) {
            const int i = (ip - kGhostX + nx) % nx;
            const int j = (jp - 1 + ny) % ny;
            const size_t s = ((size_t)k * ny + j) * nx + i;
            v.x = (T)Tsrc[s];
            v.y = (T)qsrc[s];
        }
        dst[e] = v;
    }
}

template <typename T>
__global__ void unpack_kernel(const typename Vec2<T>::type *__restrict__ src, double *__restrict__ Tdst,
                              double *__restrict__ qdst, int nx, int ny, int nz, int P, int R) {
    const size_t n = (size_t)nx * ny * nz;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % nx);
        const int j = (int)((e / nx) % ny);
        const int k = (int)(e / ((size_t)nx * ny));
        const auto v = src[((size_t)k * R + j + 1) * P + i + kGhostX];
        if (Tdst) Tdst[e] = (double)v.x;
        if (qdst) qdst[e] = (double)v.y;
    }
}

template <typename T> __global__ void convert_kernel(const double *__restrict__ s, T *__restrict__ d, size_t n) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        d[e] = (T)s[e];
}

// Column physics only, one thread per column, columns [ncol][nz].
template <typename T>
__global__ void __launch_bounds__(128) columns_kernel(const T *__restrict__ Ts, const T *__restrict__ qs,
                                                      const T *__restrict__ km, const T *__restrict__ gtab,
                                                      T *__restrict__ Tout, T *__restrict__ tend, long ncol,
                                                      int nz, T dt) {
    extern __shared__ __align__(16) unsigned char smem[];
    T *tab = reinterpret_cast<T *>(smem);
    T *cpa = tab + nz * kTab;
    T *dpa = cpa + nz * blockDim.x;
    for (int e = threadIdx.x; e < nz * kTab; e += blockDim.x) tab[e] = gtab[e];
    __syncthreads();
    const long col = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncol) return;
    const int t = threadIdx.x, nt = blockDim.x;
    const T *tc = Ts + col * nz;
    const T *qc = qs + col * nz;
    const T s = km ? km[col] : T(1);
    T cpp = 0, dpp = 0;
    for (int k = 0; k < nz; ++k) {
        const T ak = s * tab[k * kTab + TAB_AHAT];
        const T ck = s * tab[k * kTab + TAB_CHAT];
        const T m = (T(1) - ak - ck) - ak * cpp;
        const T inv = recip(m);
        cpp = ck * inv;
        dpp = (tc[k] - ak * dpp) * inv;
        cpa[k * nt + t] = cpp;
        dpa[k * nt + t] = dpp;
    }
    T x = 0, tau = 0, Etop = 1;
    for (int k = nz - 1; k >= 0; --k) {
        x = dpa[k * nt + t] - cpa[k * nt + t] * x;
        const T taub = tau + tab[k * kTab + TAB_WTAU] * qc[k];
        const T Eb = exp_neg(taub);
        const T heat = tab[k * kTab + TAB_WH] * (Etop - Eb);  // dt * H_k
        Tout[col * nz + k] = x + heat;
        if (tend) {
            tend[col * 2 * nz + k] = heat / dt;
            tend[col * 2 * nz + nz + k] = (x - tc[k]) / dt;
        }
        Etop = Eb;
        tau = taub;
    }
}

// ------------------------------------------------------------- launchers

static int cuda_fail(wx_ctx *c, cudaError_t e, const char *what) {
    c->err = std::string(what) + ": " + cudaGetErrorString(e);
    return WX_ECUDA;
}

#define WX_CK(call, what)                                   \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

static int grid_for(size_t n) {
    size_t b = (n + 255) / 256;
    return (int)(b > 65535 * 8 ? 65535 * 8 : (b == 0 ? 1 : b));
}

int launch_tables(wx_ctx *c, cudaStream_t s) {
    if (c->t_bytes == 4)
        tables_kernel<float><<<(c->nz + 127) / 128, 128, 0, s>>>(c->d_lev, c->nz, c->dt, c->kappa_h, c->S0,
                                                                 c->q_ref, (float *)c->tab);
    else
        tables_kernel<double><<<(c->nz + 127) / 128, 128, 0, s>>>(c->d_lev, c->nz, c->dt, c->kappa_h, c->S0,
                                                                  c->q_ref, (double *)c->tab);
    WX_CK(cudaGetLastError(), "tables kernel");
    return WX_OK;
}

int launch_pack(wx_ctx *c, const double *T, const double *q, void *dst, cudaStream_t s) {
    const size_t n = c->field_cells;
    if (c->t_bytes == 4)
        pack_kernel<float><<<grid_for(n), 256, 0, s>>>(T, q, (float2 *)dst, c->nx, c->ny, c->nz, c->P, c->R);
    else
        pack_kernel<double><<<grid_for(n), 256, 0, s>>>(T, q, (double2 *)dst, c->nx, c->ny, c->nz, c->P, c->R);
    WX_CK(cudaGetLastError(), "pack kernel");
    return WX_OK;
}

int launch_unpack(wx_ctx *c, const void *src, double *T, double *q, cudaStream_t s) {
    const size_t n = (size_t)c->nx * c->ny * c->nz;
    if (c->t_bytes == 4)
        unpack_kernel<float><<<grid_for(n), 256, 0, s>>>((const float2 *)src, T, q, c->nx, c->ny, c->nz, c->P,
                                                         c->R);
    else
        unpack_kernel<double><<<grid_for(n), 256, 0, s>>>((const double2 *)src, T, q, c->nx, c->ny, c->nz,
                                                          c->P, c->R);
    WX_CK(cudaGetLastError(), "unpack kernel");
    return WX_OK;
}

int launch_convert(wx_ctx *c, const double *src, void *dst, size_t n, cudaStream_t s) {
    if (c->t_bytes == 4)
        convert_kernel<float><<<grid_for(n), 256, 0, s>>>(src, (float *)dst, n);
    else
        convert_kernel<double><<<grid_for(n), 256, 0, s>>>(src, (double *)dst, n);
    WX_CK(cudaGetLastError(), "convert kernel");
    return WX_OK;
}

int launch_columns(wx_ctx *c, const void *Ts, const void *qs, const void *km, void *Tout, void *tend, long ncol,
                   cudaStream_t s) {
    if (ncol <= 0) return WX_OK;
    const int nt = 128;
    const size_t smem = (size_t)c->nz * kTab * c->t_bytes + 2 * (size_t)c->nz * nt * c->t_bytes;
    if (smem > 227 * 1024) {
        c->err = "wx_physics_columns: nz too large for the column kernel";
        return WX_EUNSUPPORTED;
    }
    const long blocks = (ncol + nt - 1) / nt;
    if (c->t_bytes == 4) {
        auto k = columns_kernel<float>;
        WX_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "smem attr");
        k<<<(unsigned)blocks, nt, smem, s>>>((const float *)Ts, (const float *)qs, (const float *)km,
                                             (const float *)c->tab, (float *)Tout, (float *)tend, ncol, c->nz,
                                             (float)c->dt);
    } else {
        auto k = columns_kernel<double>;
        WX_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "smem attr");
        k<<<(unsigned)blocks, nt, smem, s>>>((const double *)Ts, (const double *)qs, (const double *)km,
                                             (const double *)c->tab, (double *)Tout, (double *)tend, ncol,
                                             c->nz, c->dt);
    }
    WX_CK(cudaGetLastError(), "columns kernel");
    return WX_OK;
}

constexpr int kKB = 2;  // planes per TMA stage

bool cfg_fits(const wx_ctx *c, const StepCfg &cfg, int *smem_bytes) {
    const int narr = 3;
    const SmemPlan p = plan_smem(c->nz, cfg.ty, cfg.stages, kKB, c->cell_bytes, c->t_bytes, narr);
    if (smem_bytes) *smem_bytes = p.total;
    return cfg.stages >= 2 && p.total <= 227 * 1024;
}

StepCfg default_cfg(const wx_ctx *c) {
    // Prefer two CTAs per SM (<= 113 KB each) with 4 rows in FP32 / 2 in
    // FP64, and as many TMA stages as fit (up to 8); fall back to fewer rows.
    const int pref[3] = {c->t_bytes == 4 ? 4 : 2, c->t_bytes == 4 ? 2 : 1, 1};
    for (int budget : {113 * 1024, 227 * 1024}) {
        for (int ty : pref) {
            for (int st = 8; st >= 3; --st) {
                StepCfg g;
                g.ty = ty;
                g.stages = st;
                g.kb = kKB;
                int bytes = 0;
                if (cfg_fits(c, g, &bytes) && bytes <= budget) return g;
            }
        }
    }
    StepCfg g;
    g.ty = 1;
    g.stages = 2;
    return g;
}

template <typename T, int TY, bool PHYS, bool SUMS>
static int launch_step_t(wx_ctx *c, cudaStream_t s, const CUtensorMap &tm, void *out) {
    auto kern = step_kernel<T, TY, kKB, PHYS, SUMS>;
    const SmemPlan pl = plan_smem(c->nz, TY, c->cfg.stages, kKB, c->cell_bytes, c->t_bytes, PHYS ? 3 : 2);
    WX_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, pl.total), "smem attr");
    StepArgs<T> a;
    a.out = reinterpret_cast<typename Vec2<T>::type *>(out);
    a.U = (const T *)c->U;
    a.V = (const T *)c->V;
    a.kmult = (const T *)c->kmult;
    a.tab = (const T *)c->tab;
    a.status = c->d_status;
    a.partials = c->partials;
    a.nx = c->nx;
    a.ny = c->ny;
    a.nz = c->nz;
    a.P = c->P;
    a.R = c->R;
    a.dth = (T)(c->dt / c->h);
    a.dh = (T)(c->dt * c->kappa_h / (c->h * c->h));
    a.advection = (c->flags & WX_ADVECTION) ? 1 : 0;
    dim3 grid((c->nx + kTileX - 1) / kTileX, (c->ny + TY - 1) / TY);
    dim3 block(32, TY);
    kern<<<grid, block, pl.total, s>>>(tm, a, c->cfg.stages);
    WX_CK(cudaGetLastError(), "step kernel");
    return WX_OK;
}

template <typename T, bool PHYS, bool SUMS>
static int dispatch_ty(wx_ctx *c, cudaStream_t s, const CUtensorMap &tm, void *out) {
    switch (c->cfg.ty) {
        case 1: return launch_step_t<T, 1, PHYS, SUMS>(c, s, tm, out);
        case 2: return launch_step_t<T, 2, PHYS, SUMS>(c, s, tm, out);
        case 4: return launch_step_t<T, 4, PHYS, SUMS>(c, s, tm, out);
        case 8: return launch_step_t<T, 8, PHYS, SUMS>(c, s, tm, out);
        default: c->err = "unsupported tile rows"; return WX_EUNSUPPORTED;
    }
}

template <typename T>
static int dispatch_flags(wx_ctx *c, cudaStream_t s, const CUtensorMap &tm, void *out) {
    const bool phys = c->flags & WX_PHYSICS, sums = c->flags & WX_SUMS;
    if (phys && sums) return dispatch_ty<T, true, true>(c, s, tm, out);
    if (phys) return dispatch_ty<T, true, false>(c, s, tm, out);
    if (sums) return dispatch_ty<T, false, true>(c, s, tm, out);
    return dispatch_ty<T, false, false>(c, s, tm, out);
}

int launch_step(wx_ctx *c, cudaStream_t s, long *launches) {
    const int src = c->cur, dst = 1 - c->cur;
    int rc = (c->t_bytes == 4) ? dispatch_flags<float>(c, s, c->tmap[src], c->fld[dst])
                               : dispatch_flags<double>(c, s, c->tmap[src], c->fld[dst]);
    if (rc != WX_OK) return rc;
    ++*launches;
    if (c->flags & WX_SUMS) {
        const long nblk = (long)((c->nx + kTileX - 1) / kTileX) * ((c->ny + c->cfg.ty - 1) / c->cfg.ty);
        double *dst_sum = c->sums_ring + 2 * (c->sums_count % c->sums_cap);
        sums_finalize<<<1, 1024, 0, s>>>(c->partials, nblk, c->h * c->h, dst_sum);
        WX_CK(cudaGetLastError(), "sums kernel");
        ++*launches;
        ++c->sums_count;
    }
    c->cur = dst;
    return WX_OK;
}

}  // namespace wx
