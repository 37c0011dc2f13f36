// wx_step.cu -- the fused weather-step kernel and its helpers.
//
// One step n -> n+1 for every column (i, j), in two sweeps over k:
//
//   pass 1, top -> bottom (k = nz-1 .. 0)
//     dynamics: phi* = cC phi + cE phi_E + cW phi_W + cN phi_N + cS phi_S
//                      + wU_k (phi_{k+1} - phi_k) - wD_k (phi_k - phi_{k-1})
//       for phi in {T, q} (paper Eq. 1 diffusion, explicit Euler, zero flux
//       at the column ends, periodic x/y; first-order upwind advection by
//       C-grid face winds folded into cE..cS, U+ = max(U,0), U- = min(U,0):
//         cE = dh - dth Ue-,  cW = dh + dth Uw+,  cN = dh - dth Vn-,
//         cS = dh + dth Vs+,  cC = 1 - 4 dh - dth (Ue+ - Uw- + Vn+ - Vs-));
//     q^{n+1} = q* is stored at once;
//     radiation: tau accumulates from the top, H_k = S0 (2^-tau2_top -
//       2^-tau2_bot) / dz_k with tau carried in log2 units;
//     implicit vertical diffusion (I - dt L_v) x = T*: the Thomas elimination
//       run from the top, f_k = (T*_k - c_k f_{k+1}) / m_k, m_k = b_k -
//       c_k e_{k+1}, e_k = a_k / m_k (the K recurrence the paper keeps
//       sequential, Sec. 2.1);
//     the heating is folded into the back substitution: with T^{n+1}_k =
//       x_k + dt H_k and x_k = f_k - e_k x_{k-1},
//         T^{n+1}_k = F_k - e_k T^{n+1}_{k-1},  F_k = f_k + h_k + e_k h_{k-1},
//       h = dt H, so one value F_k per level is parked in shared memory.
//   pass 2, bottom -> top: T^{n+1}_k = F_k - e_k T^{n+1}_{k-1}, stored.
//
// Each field crosses HBM once per step in each direction.
#include <algorithm>
#include <cstdio>
#include <type_traits>

#include "ptx.cuh"
#include "wx_internal.cuh"

namespace wx {

// ------------------------------------------------------------ arithmetic
// Paired arithmetic on the lane's two columns: one packed f32x2 instruction
// in FP32 (sm_100+ FFMA2/FADD2/FMUL2), two scalar ones in FP64.
template <typename T> struct Pk;
template <> struct Pk<float> {
    using V = float2;
    static __device__ __forceinline__ V fma(V a, V b, V c) { return __ffma2_rn(a, b, c); }
    static __device__ __forceinline__ V mul(V a, V b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ V add(V a, V b) { return __fadd2_rn(a, b); }
    static __device__ __forceinline__ V dup(float x) { return make_float2(x, x); }
};
template <> struct Pk<double> {
    using V = double2;
    static __device__ __forceinline__ V fma(V a, V b, V c) {
        return make_double2(::fma(a.x, b.x, c.x), ::fma(a.y, b.y, c.y));
    }
    static __device__ __forceinline__ V mul(V a, V b) { return make_double2(a.x * b.x, a.y * b.y); }
    static __device__ __forceinline__ V add(V a, V b) { return make_double2(a.x + b.x, a.y + b.y); }
    static __device__ __forceinline__ V dup(double x) { return make_double2(x, x); }
};

// 2^-x: the optical depth is carried in log2 units, so exp(-tau) = 2^-tau2.
template <typename T> __device__ __forceinline__ T exp2_neg(T x);
template <> __device__ __forceinline__ float exp2_neg<float>(float x) {
    float y;  // hardware base-2 exponential (MUFU), flush-to-zero of tiny results
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));
    return y;
}
template <> __device__ __forceinline__ double exp2_neg<double>(double x) { return exp2(-x); }

template <typename T> __device__ __forceinline__ T recip(T m);
template <> __device__ __forceinline__ float recip<float>(float m) { return __frcp_rn(m); }
template <> __device__ __forceinline__ double recip<double>(double m) { return 1.0 / m; }

// Column sums of phi*dz for the lane's two columns.  FP32: dz is carried as
// hi + lo floats and every product and addition is compensated (exact
// product error, TwoSum), so the FP64 total is that of the stored FP32
// values times the FP64 dz; FP64: plain FMA accumulation.
template <typename T> struct ColSum2;
template <> struct ColSum2<float> {
    float2 s = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
    __device__ __forceinline__ void add(float2 v, float whi, float wlo) {
        const float2 w2 = make_float2(whi, whi), m1 = make_float2(-1.f, -1.f);
        const float2 p = __fmul2_rn(v, w2);
        const float2 pe = __ffma2_rn(v, make_float2(wlo, wlo), __ffma2_rn(v, w2, __fmul2_rn(p, m1)));
        const float2 s1 = __fadd2_rn(s, p);
        const float2 bp = __ffma2_rn(s, m1, s1);  // s1 - s
        const float2 sa = __ffma2_rn(bp, m1, s1); // s1 - bp
        const float2 e = __fadd2_rn(__ffma2_rn(sa, m1, s), __ffma2_rn(bp, m1, p));
        c = __fadd2_rn(c, __fadd2_rn(e, pe));
        s = s1;
    }
    __device__ __forceinline__ double total(bool va, bool vb) const {
        return (va ? (double)s.x + (double)c.x : 0.0) + (vb ? (double)s.y + (double)c.y : 0.0);
    }
};

// A float pair (s, c) standing for s + c with |c| <= ulp(s)/2: the tile's
// sums are reduced in these, with error-free TwoSum / Fast2Sum steps written
// as round-to-nearest intrinsics, so that the reduction takes no FP64
// instruction (a warp's FP64 add occupies its sub-core's FP64 unit for
// tens of cycles on this part).
struct FF {
    float s, c;
};
__device__ __forceinline__ FF ff_norm(float s, float c) {  // Fast2Sum, |s| >= |c|
    const float r = __fadd_rn(s, c);
    return FF{r, __fsub_rn(c, __fsub_rn(r, s))};
}
__device__ __forceinline__ FF ff_add(FF x, FF y) {
    const float s = __fadd_rn(x.s, y.s), bp = __fsub_rn(s, x.s);
    const float e = __fadd_rn(__fsub_rn(x.s, __fsub_rn(s, bp)), __fsub_rn(y.s, bp));  // TwoSum error
    return ff_norm(s, __fadd_rn(__fadd_rn(x.c, y.c), e));
}
// the lane's two columns as one pair (invalid columns contribute nothing)
__device__ __forceinline__ FF ff_lane(const ColSum2<float> &cs, bool va, bool vb) {
    const FF a = va ? ff_norm(cs.s.x, cs.c.x) : FF{0.f, 0.f};
    const FF b = vb ? ff_norm(cs.s.y, cs.c.y) : FF{0.f, 0.f};
    return ff_add(a, b);
}
// fixed-tree warp reduction (lane 0 ends with the warp's pair)
__device__ __forceinline__ FF ff_warp_sum(FF v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = ff_add(v, FF{__shfl_down_sync(0xffffffffu, v.s, o), __shfl_down_sync(0xffffffffu, v.c, o)});
    return v;
}

template <> struct ColSum2<double> {
    double2 s = make_double2(0.0, 0.0);
    __device__ __forceinline__ void add(double2 v, double w, double) {
        s.x = ::fma(v.x, w, s.x);
        s.y = ::fma(v.y, w, s.y);
    }
    __device__ __forceinline__ double total(bool va, bool vb) const {
        return (va ? s.x : 0.0) + (vb ? s.y : 0.0);
    }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void consumer_sync(int nthreads) {
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// ------------------------------------------------------------ step kernel
// Persistent CTAs walk tiles of 64 x TY columns (t = blockIdx.x, +gridDim.x,
// ...).  Block = TY consumer warps (lane tx owns columns 2tx, 2tx+1 of a tile
// row) + one producer warp.  The producer streams each tile's k-slabs from
// the top down (stage = KB planes x {T, q} x (TY+2) rows x 72 columns, tile
// plus a one-cell halo) through a ring of S shared-memory slots with TMA
// (full barrier: bytes landed; empty barrier: every consumer warp is done),
// and pulls slabs PF stages ahead into L2, so the next tile's loads overlap
// the current tile's stores.  KMODE 0: kappa_mult = 1 everywhere (the
// elimination coefficients come from the table); KMODE 1: per-column
// kappa_mult, eliminated on the fly; KMODE 2: table path, listed columns
// parked for the side solve.  TMF: the column state F_k lives in each
// lane's TMEM row instead of shared memory (FP32, nz <= 64), which leaves
// room for twelve consumer warps and a six-stage ring on one SM.
// One CTA per SM is the design point (persistent, shared memory and TMEM
// sized for it): the explicit minimum of 1 block lets ptxas use the whole
// register budget of the block (128 registers at 416 threads) instead of
// capping it for a second resident block and spilling.
template <typename T, int TY, int KB, int KMODE, bool PHYS, bool SUMS, bool TMF, bool RKB>
__global__ void __launch_bounds__(32 * (TY + 1), 1) step_kernel(const __grid_constant__ Members<T> ms, const int S,
                                                                const int PF) {
    static_assert(!TMF || (std::is_same<T, float>::value && KMODE != 1), "TMEM column state: FP32 table paths");
    static_assert(!RKB || (TMF && !SUMS), "RK3 stage launches: TMEM variant, no sums");
    using PK = Pk<T>;
    using V = typename PK::V;
    using R4 = Q4<T>;
    constexpr int NT = 32 * TY;           // consumer threads
    constexpr int PL = (TY + 2) * kBoxX;  // elements per staged (plane, field)
    extern __shared__ __align__(128) unsigned char smem[];

    const int tx = threadIdx.x, wy = threadIdx.y;
    const SmemPlan pl = plan_smem(ms.nz_max, TY, S, KB, (int)sizeof(T), KMODE == 1, TMF, RKB);  // e_k per column
    constexpr int PB = TY * kTileX;                                // elements per base (plane, field)
    const int BOFF = box_bytes(TY, KB, (int)sizeof(T)) / (int)sizeof(T);  // base boxes within a slot
    R4 *tab = reinterpret_cast<R4 *>(smem + pl.tab_off);
    T *ring = reinterpret_cast<T *>(smem + pl.ring_off);
    V *stF = reinterpret_cast<V *>(smem + pl.state_off);  // [nz][NT] F of the 2 columns
    V *stE = stF + ms.nz_max * NT;                         // [nz][NT] e   (KMODE 1)
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + pl.bar_off);
    uint64_t *empty = full + S;
    const int SC = pl.stage_bytes / (int)sizeof(T);
    const long total = ms.total;

    // work item w -> member index
    auto member_of = [&](long w) -> int {
        int mi = 0;
        while (mi + 1 < ms.n && w >= ms.m[mi + 1].tile0) ++mi;
        return mi;
    };

    const int tid_all = tx + 32 * wy;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(empty + S);  // TMEM base address
    if (tid_all == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], TY);
        }
        fence_mbar_init();
    }
    if (TMF && wy == 0) {  // the column state of every consumer lane lives in TMEM
        tmem_alloc(tslot, kTmemCols(TY));
        tmem_relinquish();
    }
    if (TMF) tc_fence_before();
    __syncthreads();
    if (TMF) tc_fence_after();
    // this thread's lane (its warp's lane quarter) and column group in TMEM:
    // warps w and w + 4 share a quarter and take 128 columns each
    const uint32_t trow = TMF ? *tslot + ((uint32_t)(32 * (wy & 3)) << 16) + ((uint32_t)(wy >> 2) << 7) : 0u;

    // ---------------- producer warp: stage g of a tile covers planes
    // z0 = nz - (g+1)*KB .. z0+KB-1, top of the column first
    if (wy == TY) {
        if (tx == 0 && (long)blockIdx.x < total) {
            const uint32_t tx_bytes = (uint32_t)((KB * 2 * PL + (RKB ? KB * 2 * PB : 0)) * sizeof(T));
            int slot = 0, fill = 0;
            long issued = 0;
            bool ok = true;
            // the stage sequence is (work item, stage) in order; PF stages ahead
            // of the TMA loads, L2 bulk prefetches of the same boxes
            long pw = blockIdx.x;
            int pg = 0;
            for (int ahead = 0; ahead < PF && pw < total; ++ahead) {
                const int mi = member_of(pw);
                const Member<T> &M = ms.m[mi];
                const int t = (int)(pw - M.tile0), nst = (M.a.nz + KB - 1) / KB;
                tma_prefetch_l2_4d(&M.tin, kGhostX - kBoxX0 + (t % M.gx) * kTileX, (t / M.gx) * TY, 0,
                                   M.a.nz - (pg + 1) * KB);
                if (++pg == nst) {
                    pg = 0;
                    pw += gridDim.x;
                }
            }
            for (long w = blockIdx.x; w < total && ok; w += gridDim.x) {
                const int mi = member_of(w);
                const Member<T> &M = ms.m[mi];
                prefetch_tmap(&M.tin);
                const int t = (int)(w - M.tile0), nz = M.a.nz, nst = (nz + KB - 1) / KB;
                const int x0 = kGhostX - kBoxX0 + (t % M.gx) * kTileX;  // multiple of 4 elements
                const int y0 = (t / M.gx) * TY;
                for (int g = 0; g < nst; ++g) {
                    if (PF > 0 && pw < total) {
                        const int pmi = member_of(pw);
                        const Member<T> &PM = ms.m[pmi];
                        const int pt = (int)(pw - PM.tile0), pnst = (PM.a.nz + KB - 1) / KB;
                        tma_prefetch_l2_4d(&PM.tin, kGhostX - kBoxX0 + (pt % PM.gx) * kTileX, (pt / PM.gx) * TY, 0,
                                           PM.a.nz - (pg + 1) * KB);
                        if (++pg == pnst) {
                            pg = 0;
                            pw += gridDim.x;
                        }
                    }
                    if (issued >= S && !mbar_wait_bounded(&empty[slot], (uint32_t)((fill - 1) & 1))) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[slot], tx_bytes);
                    tma_load_4d(ring + slot * SC, &M.tin, &full[slot], x0, y0, 0, nz - (g + 1) * KB);
                    if (RKB)  // phi^n of the tile's interior, same planes
                        tma_load_4d(ring + slot * SC + BOFF, &M.tbase, &full[slot], x0 + kBoxX0, y0 + 1, 0,
                                    nz - (g + 1) * KB);
                    ++issued;
                    if (++slot == S) {
                        slot = 0;
                        ++fill;
                    }
                }
            }
            if (!ok) atomicOr(ms.status, ST_TIMEOUT);
            // keep this thread until its last copy into every slot has landed
            for (int s = 0; s < S && s < issued; ++s)
                (void)mbar_wait_bounded(&full[s], (uint32_t)(((issued - 1 - s) / S) & 1));
        }
        return;
    }

    // ---------------- consumers: two adjacent columns per lane
    // stores into a member's new state (range-checked in the bounds-checked
    // build, plain stores otherwise)
    auto put = [&](const StepArgs<T> &ar, T *p, T v) {
        if (WX_IN(p - ar.out, ar.out_n, ar.status)) *p = v;
    };
    auto put2 = [&](const StepArgs<T> &ar, T *p, V v) {
        if (WX_IN(p - ar.out + 1, ar.out_n, ar.status)) *reinterpret_cast<V *>(p) = v;
    };
    const int tid = tx + 32 * wy;
    const int ctr = (wy + 1) * kBoxX + kBoxX0 + 2 * tx;  // column pair in a staged plane (8-byte aligned)
    const T zero = T(0);
    const V m1 = PK::dup(T(-1));
    int slot = 0;
    uint32_t par = 0;
    bool ok = true;
    int cur_member = -1;

    // face winds of a tile's two columns (a, b): Ue, Uw, Vn, Vs each
    struct Winds {
        T v[8];
    };
    auto load_winds = [&](long w) -> Winds {
        Winds wd;
        const Member<T> &M = ms.m[member_of(w)];
        const int t = (int)(w - M.tile0);
        const int nx = M.a.nx, ny = M.a.ny;
        const int i0 = (t % M.gx) * kTileX + 2 * tx, j = (t / M.gx) * TY + wy;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const bool v = (i0 + c < nx) && (j < ny) && M.a.advection &&
                           WX_IN((long long)j * nx + i0 + c, (long long)nx * ny, M.a.status);
            const int ic = v ? i0 + c : 0, jc = v ? j : 0;
            wd.v[4 * c + 0] = v ? M.a.U[(size_t)jc * nx + ic] : T(0);
            const T *uw = (ic == 0 && M.a.Uw0) ? M.a.Uw0 + jc : M.a.U + (size_t)jc * nx + (ic == 0 ? nx - 1 : ic - 1);
            const T *vs = (jc == 0 && M.a.Vs0) ? M.a.Vs0 + ic : M.a.V + (size_t)(jc == 0 ? ny - 1 : jc - 1) * nx + ic;
            wd.v[4 * c + 1] = v ? *uw : T(0);
            wd.v[4 * c + 2] = v ? M.a.V[(size_t)jc * nx + ic] : T(0);
            wd.v[4 * c + 3] = v ? *vs : T(0);
        }
        return wd;
    };
    Winds wnext = load_winds((long)blockIdx.x < total ? (long)blockIdx.x : 0);

    for (long w = blockIdx.x; w < total; w += gridDim.x) {
        const int mi = member_of(w);
        const StepArgs<T> a = ms.m[mi].a;
        const int nx = a.nx, ny = a.ny, nz = a.nz;
        const int gx = ms.m[mi].gx, gy = ms.m[mi].gy;
        const int n_st = (nz + KB - 1) / KB;
        const size_t lev = (size_t)2 * a.R * a.P;  // elements between levels
        const size_t fld = (size_t)a.R * a.P;      // T plane -> q plane
        if (mi != cur_member) {  // stage the member's per-level table
            consumer_sync(NT);
            for (int e = tid; e < kTabRec * nz; e += NT) tab[e] = a.tab[e];
            consumer_sync(NT);
            cur_member = mi;
        }
        const R4 *tA = tab + REC_A * nz, *tB = tab + REC_B * nz, *tC = tab + REC_C * nz, *tD = tab + REC_D * nz,
                 *tE = tab + REC_E * nz, *tF = tab + REC_F * nz;
        const int t = (int)(w - ms.m[mi].tile0);
        const int bx = t % gx, by = t / gx;
        const int i0 = bx * kTileX + 2 * tx, j = by * TY + wy;
        const bool va = (i0 < nx) && (j < ny), vb = (i0 + 1 < nx) && (j < ny);
        // tile kind: 0 inner (whole 64 x TY columns, no edge), 1 a whole
        // border tile (paired stores plus the ghost copies of its edge
        // lanes and rows), 2 a ragged tile (masked stores plus ghost copies)
        const bool ragged = (bx == gx - 1 && nx % kTileX) || (by == gy - 1 && ny % TY);
        const int kind = ragged ? 2 : ((bx == 0 || bx == gx - 1 || by == 0 || by == gy - 1) ? 1 : 0);
        // this lane's ghost duties: column 0 (x), column nx-1 (x or y)
        const bool gc0 = va && i0 == 0, gclx = va && i0 == nx - 1, gcly = vb && i0 + 1 == nx - 1;
        const bool gwarp = __any_sync(0xffffffffu, gc0 || gclx || gcly);  // warp-uniform
        const size_t rowoff = (size_t)(j + 1) * a.P + (i0 + kGhostX);

        // per-column coefficients of the horizontal operator, paired (a, b)
        const Winds wc = wnext;
        if (w + (long)gridDim.x < total) wnext = load_winds(w + gridDim.x);  // in flight during the tile
        V cC, cE, cW, cN, cS, km;
        int fl[2];
        {
            T c5[2][5], k1[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const T ue = wc.v[4 * c], uw = wc.v[4 * c + 1], vn = wc.v[4 * c + 2], vs = wc.v[4 * c + 3];
                c5[c][1] = a.dh - a.dth * fmin(ue, zero);
                c5[c][2] = a.dh + a.dth * fmax(uw, zero);
                c5[c][3] = a.dh - a.dth * fmin(vn, zero);
                c5[c][4] = a.dh + a.dth * fmax(vs, zero);
                c5[c][0] = T(1) - T(4) * a.dh -
                           a.dth * (fmax(ue, zero) - fmin(uw, zero) + fmax(vn, zero) - fmin(vs, zero));
                const bool v = c ? vb : va;
                const bool inb = v && WX_IN((long long)j * nx + i0 + c, (long long)nx * ny, a.status);
                k1[c] = (KMODE == 1 && a.kmult && v && inb) ? a.kmult[(size_t)j * nx + i0 + c] : T(1);
                fl[c] = (KMODE == 2 && v && a.flag_idx && inb) ? a.flag_idx[(size_t)j * nx + i0 + c] : -1;
            }
            cC = V{c5[0][0], c5[1][0]};
            cE = V{c5[0][1], c5[1][1]};
            cW = V{c5[0][2], c5[1][2]};
            cN = V{c5[0][3], c5[1][3]};
            cS = V{c5[0][4], c5[1][4]};
            km = V{k1[0], k1[1]};
        }

        // ------------- pass 1 (top down)
        if (ok) ok = mbar_wait_bounded(&full[slot], par);
        // plane (sub-plane s, field f) of the slot: ring + slot*SC + (s*2 + f)*PL
        const T *p0 = ring + slot * SC + ((KB - 1) * 2) * PL;  // top plane of the tile
        V curT = *reinterpret_cast<const V *>(p0 + ctr);
        V curQ = *reinterpret_cast<const V *>(p0 + PL + ctr);
        V prvT = curT, prvQ = curQ;
        V tau = PK::dup(T(0)), Et = PK::dup(T(1));
        V f_up = PK::dup(T(0)), h_up = PK::dup(T(0)), e_up = PK::dup(T(0));  // level k+1
        V chk = PK::dup(T(0));
        ColSum2<T> sumQ, sumT;
        // A level's new pair of field f into the new state (kind as above),
        // then its copies into the grid's periodic ghost ring, addressed from
        // the store: column 0 -> ghost column nx, column nx-1 -> ghost column
        // -1, row 0 -> ghost row ny+1, row ny-1 -> ghost row 0.  (A block of
        // a decomposed grid gets its ghost lines from the halo exchange that
        // follows the step; these copies are then overwritten.)
        auto emit = [&](auto kind_tag, int k, int f, V v) {
            constexpr int KIND = decltype(kind_tag)::value;
            T *dst = a.out + (size_t)k * lev + (size_t)f * fld + rowoff;
            if (KIND != 2) {
                put2(a, dst, v);
            } else {
                if (va) put(a, dst, v.x);
                if (vb) put(a, dst + 1, v.y);
            }
            if (KIND == 0) return;
            if (gwarp) {
                if (gc0) put(a, dst + nx, v.x);
                if (gclx) put(a, dst - nx, v.x);
                if (gcly) put(a, dst + 1 - nx, v.y);
            }
            for (int r = 0; r < 2; ++r) {  // warp-uniform; both rows when ny = 1
                if (j != (r == 0 ? 0 : ny - 1)) continue;
                T *g = r == 0 ? dst + (size_t)ny * a.P : dst - (size_t)ny * a.P;
                if (KIND != 2) {
                    put2(a, g, v);
                } else {
                    if (va) put(a, g, v.x);
                    if (vb) put(a, g + 1, v.y);
                }
            }
        };
        // F_k of the lane's two columns: its TMEM lane, or shared memory
        auto putF = [&](int k, V v) {
            if constexpr (TMF) {
                if (WX_IN(2 * k + 1, 128, a.status)) tmem_st2(trow + 2 * k, v.x, v.y);  // k is warp-uniform
            } else {
                stF[k * NT + tid] = v;
            }
        };

        // phi* for one field at level k: two short FMA chains, summed
        auto stencil = [&](const T *pf, V cur, V prv, V nxt, V cCk, V wu, V wd) -> V {
            const V n = *reinterpret_cast<const V *>(pf + ctr + kBoxX);
            const V s = *reinterpret_cast<const V *>(pf + ctr - kBoxX);
            const T e = pf[ctr + 2], w = pf[ctr - 1];
            V c1 = PK::fma(cN, n, PK::mul(cCk, cur));
            c1.x = ::fma(cE.x, cur.y, c1.x);
            c1.y = ::fma(cE.y, e, c1.y);
            V c2 = PK::fma(wd, nxt, PK::fma(wu, prv, PK::mul(cS, s)));
            c2.x = ::fma(cW.x, w, c2.x);
            c2.y = ::fma(cW.y, cur.x, c2.y);
            return PK::add(c1, c2);
        };

        // one level; EDGE selects the masked store path with ghost copies
        auto level = [&](auto edge_tag, int k, const T *pk, const T *pb, V nT, V nQ) {
            constexpr bool EDGE = decltype(edge_tag)::value == 2;  // masked (ragged) tile
            const R4 A = tA[k], B = tB[k];
            const V wu = V{A.x, A.y}, wd = V{A.z, A.w};
            const V cCk = PK::add(cC, V{B.x, B.y});
            V Ts = stencil(pk, curT, prvT, nT, cCk, wu, wd);
            V Qs = stencil(pk + PL, curQ, prvQ, nQ, cCk, wu, wd);
            if (RKB) {  // RK3 stage: phi^n + (E - phi_s), E = phi_s + c dt L(phi_s)
                const V bT = *reinterpret_cast<const V *>(pb), bQ = *reinterpret_cast<const V *>(pb + PB);
                Ts = PK::add(bT, PK::fma(curT, m1, Ts));
                Qs = PK::add(bQ, PK::fma(curQ, m1, Qs));
            }
            prvT = curT;
            prvQ = curQ;
            curT = nT;
            curQ = nQ;

            // q^{n+1} = q*
            emit(edge_tag, k, 1, Qs);
            const V Qm = EDGE ? V{va ? Qs.x : T(0), vb ? Qs.y : T(0)} : Qs;
            if (SUMS)
                sumQ.add(Qm, tF[k].z, tF[k].w);
            else
                chk = PK::add(chk, Qm);

            if (PHYS) {
                const R4 C = tC[k];
                // radiation from the top: h = dt H_k = wH (E_top - E_bot)
                const V tb = PK::fma(V{B.z, B.w}, Qs, tau);
                const V Eb = V{exp2_neg(tb.x), exp2_neg(tb.y)};
                const V hk = PK::mul(V{C.x, C.y}, PK::fma(Eb, m1, Et));
                Et = Eb;
                tau = tb;
                // elimination from the top
                V fk, ek;
                if (KMODE != 1) {
                    const R4 D = tD[k];
                    fk = PK::mul(PK::fma(V{C.z, C.w}, f_up, Ts), V{D.x, D.y});
                    ek = V{D.z, D.w};
                } else {
                    const R4 E = tE[k];
                    const V ak = PK::mul(km, PK::dup(E.x));
                    const V nck = PK::mul(km, PK::dup(-E.y));  // -c_k
                    // m = (1 - a - c) - c e_{k+1}
                    const V m = PK::fma(nck, e_up, PK::add(PK::fma(ak, m1, PK::dup(T(1))), nck));
                    const V inv = V{recip(m.x), recip(m.y)};
                    fk = PK::mul(PK::fma(nck, f_up, Ts), inv);
                    ek = PK::mul(ak, inv);
                    stE[k * NT + tid] = PK::mul(ek, m1);
                }
                if (KMODE == 2) {  // listed columns: T* and dt*H for the side solve, [k][2][n]
                    float *sd = a.side + (size_t)k * 2 * a.n_list;
                    if (fl[0] >= 0 && WX_IN(fl[0], a.n_list, a.status)) {
                        sd[fl[0]] = (float)Ts.x;
                        sd[a.n_list + fl[0]] = (float)hk.x;
                    }
                    if (fl[1] >= 0 && WX_IN(fl[1], a.n_list, a.status)) {
                        sd[fl[1]] = (float)Ts.y;
                        sd[a.n_list + fl[1]] = (float)hk.y;
                    }
                }
                // F_{k+1} = f_{k+1} + h_{k+1} + e_{k+1} h_k  (complete now)
                if (k + 1 < nz) putF(k + 1, PK::fma(e_up, hk, PK::add(f_up, h_up)));
                f_up = fk;
                h_up = hk;
                e_up = ek;
            } else {
                putF(k, Ts);
            }
        };

        // stage g holds levels z0 .. z0+KB-1 (sub-planes 0..KB-1), z0 =
        // nz - KB(g+1); the level below z0 is the top sub-plane of stage g+1
        auto run_pass1 = [&](auto edge_tag) {
            for (int g = 0; g < n_st; ++g) {
                const T *pa = ring + slot * SC;
                const int nslot = (slot + 1 == S) ? 0 : slot + 1;
                const uint32_t npar = (nslot == 0) ? (par ^ 1u) : par;
                const int z0 = nz - (g + 1) * KB;
#pragma unroll
                for (int s = KB - 1; s >= 0; --s) {
                    const int k = z0 + s;
                    if (k < 0) continue;  // below the column (last stage only)
                    V nT = curT, nQ = curQ;
                    if (s > 0) {
                        if (k >= 1) {
                            nT = *reinterpret_cast<const V *>(pa + (s - 1) * 2 * PL + ctr);
                            nQ = *reinterpret_cast<const V *>(pa + (s - 1) * 2 * PL + PL + ctr);
                        }
                    } else if (k >= 1) {
                        if (ok) ok = mbar_wait_bounded(&full[nslot], npar);
                        const T *pn = ring + nslot * SC + (KB - 1) * 2 * PL;
                        nT = *reinterpret_cast<const V *>(pn + ctr);
                        nQ = *reinterpret_cast<const V *>(pn + PL + ctr);
                    }
                    level(edge_tag, k, pa + s * 2 * PL, pa + BOFF + (s * 2 * TY + wy) * kTileX + 2 * tx, nT, nQ);
                }
                __syncwarp();
                if (tx == 0) mbar_arrive(&empty[slot]);
                slot = nslot;
                par = npar;
            }
        };
        if (kind == 0)
            run_pass1(std::integral_constant<int, 0>{});
        else if (kind == 1)
            run_pass1(std::integral_constant<int, 1>{});
        else
            run_pass1(std::integral_constant<int, 2>{});
        if (PHYS) putF(0, PK::add(f_up, h_up));  // F_0 = f_0 + h_0

        // ------------- pass 2 (bottom up): T^{n+1}_k = F_k - e_k T^{n+1}_{k-1}
        V Tprev = PK::dup(T(0));
        // listed columns (KMODE 2 with physics) are finished by the side
        // solve, which sums their final T itself: their table-path T stays
        // out of the sums
        constexpr bool SIDE = KMODE == 2 && PHYS;
        const V lmask = V{(SIDE && fl[0] >= 0) ? T(0) : T(1), (SIDE && fl[1] >= 0) ? T(0) : T(1)};
        auto back = [&](auto edge_tag, int k, V tn) {
            constexpr bool EDGE = decltype(edge_tag)::value == 2;  // masked (ragged) tile
            const R4 Fr = tF[k];
            if (PHYS) {
                const V ne = (KMODE != 1) ? V{Fr.x, Fr.y} : stE[k * NT + tid];
                tn = PK::fma(ne, Tprev, tn);
                Tprev = tn;
            }
            emit(edge_tag, k, 0, tn);
            const V tm = EDGE ? V{va ? tn.x : T(0), vb ? tn.y : T(0)} : tn;
            if (SUMS)
                sumT.add(SIDE ? PK::mul(tm, lmask) : tm, Fr.z, Fr.w);
            else
                chk = PK::add(chk, tm);
        };
        auto run_pass2 = [&](auto edge_tag) {
            if constexpr (TMF) {
                // F of 8 levels per TMEM load (16 columns of the lane)
                tmem_wait_st();
                for (int k0 = 0; k0 < nz; k0 += 8) {
                    float fv[16];
                    tmem_ld16(trow + 2 * k0, fv);
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (k0 + u < nz) back(edge_tag, k0 + u, V{fv[2 * u], fv[2 * u + 1]});
                }
            } else {
#pragma unroll 4
                for (int k = 0; k < nz; ++k) back(edge_tag, k, stF[k * NT + tid]);
            }
        };
        if (kind == 0)
            run_pass2(std::integral_constant<int, 0>{});
        else if (kind == 1)
            run_pass2(std::integral_constant<int, 1>{});
        else
            run_pass2(std::integral_constant<int, 2>{});

        if constexpr (SUMS && std::is_same<T, float>::value) {
            // deterministic per-tile reduction in float pairs: the lane's
            // columns, a warp tree, then a fixed tree over the warps in warp 0
            __shared__ FF redf[2 * TY];
            const FF pq = ff_warp_sum(ff_lane(sumQ, va, vb)), pt = ff_warp_sum(ff_lane(sumT, va, vb));
            if (tx == 0) {
                redf[2 * wy] = pq;
                redf[2 * wy + 1] = pt;
            }
            consumer_sync(NT);
            if (wy == 0) {
                FF q = tx < TY ? redf[2 * tx] : FF{0.f, 0.f}, tt = tx < TY ? redf[2 * tx + 1] : FF{0.f, 0.f};
                q = ff_warp_sum(q);
                tt = ff_warp_sum(tt);
                if (tx == 0) {
                    if (!isfinite(q.s) || !isfinite(q.c) || !isfinite(tt.s) || !isfinite(tt.c))
                        atomicOr(a.status, ST_NONFINITE);
                    a.partials[2 * (size_t)t] = (double)q.s + (double)q.c;
                    a.partials[2 * (size_t)t + 1] = (double)tt.s + (double)tt.c;
                }
            }
            consumer_sync(NT);
        } else if constexpr (SUMS) {
            double mT = sumT.total(va, vb), mQ = sumQ.total(va, vb);
            if ((va || vb) && (!isfinite(mT) || !isfinite(mQ))) atomicOr(a.status, ST_NONFINITE);
            // deterministic per-tile reduction: warp tree, then warps in order
            __shared__ double red[2 * TY];
            mT = warp_sum(mT);
            mQ = warp_sum(mQ);
            if (tx == 0) {
                red[2 * wy] = mQ;
                red[2 * wy + 1] = mT;
            }
            consumer_sync(NT);
            if (tid == 0) {
                double q = 0.0, tt = 0.0;
                for (int w = 0; w < TY; ++w) {
                    q += red[2 * w];
                    tt += red[2 * w + 1];
                }
                a.partials[2 * (size_t)t] = q;
                a.partials[2 * (size_t)t + 1] = tt;
            }
            consumer_sync(NT);
        } else {
            if (!isfinite(chk.x) || !isfinite(chk.y))
                atomicOr(a.status, ST_NONFINITE);  // edge tiles tallied only their valid columns
        }
    }
    if (!ok && tx == 0) atomicOr(ms.status, ST_TIMEOUT);
    if constexpr (TMF) {  // every consumer is done with its lane: free the columns
        tc_fence_before();
        consumer_sync(NT);
        tc_fence_after();
        if (wy == 0) tmem_dealloc(*tslot, kTmemCols(TY));
    }
}

// Fixed-order FP64 reduction of the per-tile partials (and of the side
// solve's energy corrections) into one ring entry.  Block b reduces a fixed
// chunk with a fixed tree and parks its result; the last block to finish
// (ticket) adds the parked results in block order, so the total does not
// depend on scheduling.
constexpr int kFinBlocks = 64;
__global__ void __launch_bounds__(256) sums_finalize(const double *__restrict__ part, long nblk,
                                                     const double *__restrict__ corr, long ncorr, double h2,
                                                     double *__restrict__ park, unsigned *__restrict__ ticket,
                                                     double *__restrict__ ring, long long *__restrict__ count,
                                                     int cap) {
    __shared__ double sq[8], st[8];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long per = (nblk + gridDim.x - 1) / gridDim.x, perc = (ncorr + gridDim.x - 1) / gridDim.x;
    const long b0 = blockIdx.x * per, b1 = min(nblk, b0 + per);
    const long c0 = blockIdx.x * perc, c1 = min(ncorr, c0 + perc);
    double q = 0.0, t = 0.0;
    for (long b = b0 + threadIdx.x; b < b1; b += blockDim.x) {
        q += part[2 * b];
        t += part[2 * b + 1];
    }
    for (long b = c0 + threadIdx.x; b < c1; b += blockDim.x) t += corr[b];
    // fixed trees: within each warp, then over the block's eight warps
    q = warp_sum(q);
    t = warp_sum(t);
    if (lane == 0) {
        sq[warp] = q;
        st[warp] = t;
    }
    __syncthreads();
    if (warp == 0) {
        q = lane < 8 ? sq[lane] : 0.0;
        t = lane < 8 ? st[lane] : 0.0;
        q = warp_sum(q);
        t = warp_sum(t);
        if (lane == 0) {
            park[2 * blockIdx.x] = q;
            park[2 * blockIdx.x + 1] = t;
            __threadfence();
            last = atomicAdd(ticket, 1u) == gridDim.x - 1;
        }
    }
    __syncthreads();
    if (!last) return;
    // the last block: the parked block results in a fixed tree (block b in
    // lane b % 32 of warp b / 32), then the warps in order
    __threadfence();
    q = 0.0;
    t = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        q += ((volatile double *)park)[2 * b];
        t += ((volatile double *)park)[2 * b + 1];
    }
    q = warp_sum(q);
    t = warp_sum(t);
    __syncthreads();
    if (lane == 0) {
        sq[warp] = q;
        st[warp] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double Q = 0.0, Tt = 0.0;
        for (int w = 0; w < 8; ++w) {
            Q += sq[w];
            Tt += st[w];
        }
        // the ring slot comes from a device counter, so a captured graph
        // replays into the next slots
        const long long n = *count;
        double *dst = ring + 2 * (n % cap);
        dst[0] = h2 * Q;
        dst[1] = h2 * Tt;
        *count = n + 1;
        *ticket = 0u;  // ready for the next step
    }
}

// Per-level table from FP64 dz, kappa_lev, alpha.  One thread: the
// kappa_mult = 1 column's elimination from the top is a recurrence in k.
template <typename T>
__global__ void tables_kernel(const double *lev, int nz, double dt, double kappa_h, double S0, double q_ref,
                              Q4<T> *tab) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const double *dz = lev, *kl = lev + nz, *al = lev + 2 * nz;
    const double log2e = 1.4426950408889634074;
    double e_up = 0.0;
    for (int k = nz - 1; k >= 0; --k) {
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
        const double m = (1.0 - ah - ch) - ch * e_up;  // kappa_mult = 1 pivot, from the top
        const double e = ah / m;
        e_up = e;
        tab[REC_A * nz + k] = Q4<T>{(T)wU, (T)wU, (T)wD, (T)wD};
        const double wt2 = al[k] * dz[k] * log2e / q_ref;
        tab[REC_B * nz + k] = Q4<T>{(T)(-(wU + wD)), (T)(-(wU + wD)), (T)wt2, (T)wt2};
        const double wH = dt * S0 / dz[k];
        tab[REC_C * nz + k] = Q4<T>{(T)wH, (T)wH, (T)(-ch), (T)(-ch)};
        tab[REC_D * nz + k] = Q4<T>{(T)(1.0 / m), (T)(1.0 / m), (T)e, (T)e};
        tab[REC_E * nz + k] = Q4<T>{(T)ah, (T)ch, (T)dz[k], (T)0};
        const T dz_hi = (T)dz[k];
        tab[REC_F * nz + k] = Q4<T>{(T)(-e), (T)(-e), dz_hi, (T)(dz[k] - (double)dz_hi)};
    }
}

// Column physics only, one thread per column, columns [ncol][nz]: the
// forward Thomas sweep of the implicit vertical diffusion and the
// optical-depth scan from the top (same definitions as the step).
template <typename T>
__global__ void __launch_bounds__(128) columns_kernel(const T *__restrict__ Ts, const T *__restrict__ qs,
                                                      const T *__restrict__ km, const Q4<T> *__restrict__ gtab,
                                                      T *__restrict__ Tout, T *__restrict__ tend, long ncol,
                                                      int nz, T dt) {
    extern __shared__ __align__(128) unsigned char smem[];
    Q4<T> *tab = reinterpret_cast<Q4<T> *>(smem);
    T *cpa = reinterpret_cast<T *>(tab + kTabRec * nz);
    T *dpa = cpa + nz * blockDim.x;
    for (int e = threadIdx.x; e < kTabRec * nz; e += blockDim.x) tab[e] = gtab[e];
    __syncthreads();
    const long col = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncol) return;
    const int t = threadIdx.x, nt = blockDim.x;
    const T *tc = Ts + col * nz;
    const T *qc = qs + col * nz;
    const T s = km ? km[col] : T(1);
    const Q4<T> *tB = tab + REC_B * nz, *tC = tab + REC_C * nz, *tE = tab + REC_E * nz;
    ThomasSweep<T> fw;
    for (int k = 0; k < nz; ++k) {
        cpa[k * nt + t] = fw.level(-s * tE[k].x, -s * tE[k].y, tc[k]);
        dpa[k * nt + t] = fw.d;
    }
    T x = 0, tau = 0, Etop = 1;
    for (int k = nz - 1; k >= 0; --k) {
        x = dpa[k * nt + t] - cpa[k * nt + t] * x;
        const T taub = tau + tB[k].z * qc[k];
        const T Eb = exp2_neg(taub);
        const T heat = tC[k].x * (Etop - Eb);  // dt * H_k
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

#define WX_CK(call, what)                                     \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

static int grid_for(size_t n) {
    size_t b = (n + 255) / 256;
    return (int)(b > 65535 * 8 ? 65535 * 8 : (b == 0 ? 1 : b));
}

// Tables for another step length (the RK3 stages), written to dst.
int launch_tables_dt(wx_ctx *c, double dt, void *dst, cudaStream_t s) {
    if (c->t_bytes == 4)
        tables_kernel<float><<<1, 32, 0, s>>>(c->d_lev, c->nz, dt, c->kappa_h, c->S0, c->q_ref, (Q4<float> *)dst);
    else
        tables_kernel<double><<<1, 32, 0, s>>>(c->d_lev, c->nz, dt, c->kappa_h, c->S0, c->q_ref, (Q4<double> *)dst);
    WX_CK(cudaGetLastError(), "tables kernel");
    return WX_OK;
}

int launch_tables(wx_ctx *c, cudaStream_t s) {
    if (c->t_bytes == 4)
        tables_kernel<float><<<1, 32, 0, s>>>(c->d_lev, c->nz, c->dt, c->kappa_h, c->S0, c->q_ref,
                                              (Q4<float> *)c->tab);
    else
        tables_kernel<double><<<1, 32, 0, s>>>(c->d_lev, c->nz, c->dt, c->kappa_h, c->S0, c->q_ref,
                                               (Q4<double> *)c->tab);
    WX_CK(cudaGetLastError(), "tables kernel");
    return WX_OK;
}

int launch_columns(wx_ctx *c, const void *Ts, const void *qs, const void *km, void *Tout, void *tend, long ncol,
                   cudaStream_t s) {
    if (ncol <= 0) return WX_OK;
    const int nt = 128;
    const size_t smem = (size_t)c->nz * kTabRec * 4 * c->t_bytes + 2 * (size_t)c->nz * nt * c->t_bytes;
    if (smem > 227 * 1024) {
        c->err = "wx_physics_columns: nz too large for the column kernel";
        return WX_EUNSUPPORTED;
    }
    const long blocks = (ncol + nt - 1) / nt;
    if (c->t_bytes == 4) {
        auto k = columns_kernel<float>;
        WX_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "smem attr");
        k<<<(unsigned)blocks, nt, smem, s>>>((const float *)Ts, (const float *)qs, (const float *)km,
                                             (const Q4<float> *)c->tab, (float *)Tout, (float *)tend, ncol, c->nz,
                                             (float)c->dt);
    } else {
        auto k = columns_kernel<double>;
        WX_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "smem attr");
        k<<<(unsigned)blocks, nt, smem, s>>>((const double *)Ts, (const double *)qs, (const double *)km,
                                             (const Q4<double> *)c->tab, (double *)Tout, (double *)tend, ncol,
                                             c->nz, c->dt);
    }
    WX_CK(cudaGetLastError(), "columns kernel");
    return WX_OK;
}


// FP32 storage (WX_MIXED and WX_F32) with listed kappa_mult != 1 columns:
// table path for every column, side solve for the listed ones (in FP64 for
// the weakly dominant columns of WX_MIXED, in FP32 otherwise).  FP64
// storage with kappa_mult eliminates per column on the fly.
static bool mixed(const wx_ctx *c) { return (c->dtype == WX_MIXED || c->dtype == WX_F32) && c->n_list > 0; }
static bool per_col(const wx_ctx *c) { return c->kmult != nullptr && c->dtype == WX_F64; }
// The TMEM column-state variant: FP32 storage (table paths) with columns of
// at most kTmemMaxNz levels, at the tile heights it is built for.
static bool tmem_nz(int t_bytes, int nz, bool pc) { return t_bytes == 4 && !pc && nz <= kTmemMaxNz; }
static bool tmem_shape(int ty, int kb) { return ty == 12 && kb == 4; }
static bool use_tmem(const wx_ctx *c, const StepCfg &g) {
    return tmem_nz(c->t_bytes, c->nz, per_col(c)) && tmem_shape(g.ty, g.kb);
}

bool cfg_fits(const wx_ctx *c, const StepCfg &cfg, int *smem_bytes) {
    const bool tm = use_tmem(c, cfg);
    const SmemPlan p = plan_smem(c->nz, cfg.ty, cfg.stages, cfg.kb, c->t_bytes, per_col(c), tm);
    if (smem_bytes) *smem_bytes = p.total;
    if (cfg.ty == 12 && !tm) return false;  // twelve-row tiles exist with TMEM column state only
    // the per-SM budget: ctas_per_sm CTAs plus 1 KB runtime reserve each;
    // with TMEM column state, their columns within the SM's 512
    return cfg.stages >= 3 && (cfg.kb == 2 || cfg.kb == 4) && cfg.ctas_per_sm >= 1 && p.total <= 227 * 1024 &&
           cfg.ctas_per_sm * (p.total + 1024) <= 228 * 1024 &&
           (!tm || cfg.ctas_per_sm * (int)kTmemCols(cfg.ty) <= 512);
}

StepCfg default_cfg(const wx_ctx *c) {
    // The TMA unit of an SM completes boxes at a roughly fixed rate, so big
    // boxes (4 planes) and tall tiles come first; then the most resident
    // consumer warps per SM (capped at 16), then the deeper ring (3..6
    // slots: measured at the paper grid, a ring that leaves the SM less
    // than ~30 KB of L1 -- 7 slots of twelve-row boxes, 231 KB -- runs 40%
    // slower than 6).
    StepCfg best;
    best.ty = 1;
    best.stages = 3;
    best.kb = 2;
    best.ctas_per_sm = 1;
    long best_score = -1;
    for (int kb : {2, 4}) {
        for (int ty : {1, 2, 4, 8, 12}) {
            if (ty == 12 && !tmem_nz(c->t_bytes, c->nz, per_col(c))) continue;
            for (int st = 6; st >= 3; --st) {
                StepCfg g;
                g.ty = ty;
                g.stages = st;
                g.kb = kb;
                int bytes = 0;
                g.ctas_per_sm = 1;
                if (!cfg_fits(c, g, &bytes)) continue;
                g.ctas_per_sm = std::min(228 * 1024 / (bytes + 1024), 2048 / (32 * (ty + 1)));
                if (use_tmem(c, g)) g.ctas_per_sm = std::min(g.ctas_per_sm, 512 / (int)kTmemCols(ty));
                const int warps = std::min(g.ctas_per_sm * ty, 16);
                if (!cfg_fits(c, g, nullptr)) continue;
                const long box = (long)kb * 2 * (ty + 2) * kBoxX * c->t_bytes;  // both fields
                const long score = ((box >= 16384) ? 1L << 40 : 0) + ((long)warps << 20) + ((long)ty << 10) + st;
                if (score > best_score) {
                    best = g;
                    best_score = score;
                }
            }
        }
    }
    best.prefetch = 0;
    return best;
}

// ------------------------------------------------------------- batches
// A batch = the members one launch steps (one context, or an ensemble's
// members), with the launch configuration of its owner.
template <typename T> static void fill_member(const wx_ctx *c, Member<T> &M, long tile0, int ty) {
    const bool stage = c->stage_in >= 0;  // one RK3 stage: its buffers, step and table
    const int src = stage ? c->stage_in : c->cur, dst = stage ? c->stage_out : 1 - c->cur;
    const double dt = stage ? c->stage_dt : c->dt;
    M.tin = c->tmap[src];
    if (stage && c->stage_base >= 0) M.tbase = c->tmap_rkbase;
    StepArgs<T> &a = M.a;
    a.out = reinterpret_cast<T *>(c->fld[dst]);
    a.U = (const T *)c->U;
    a.V = (const T *)c->V;
    a.kmult = (const T *)c->kmult;
    a.tab = (const Q4<T> *)(stage ? c->stage_tab : c->tab);
    a.status = c->d_status;
    a.partials = c->partials;
    a.nx = c->nx;
    a.ny = c->ny;
    a.nz = c->nz;
    a.P = c->P;
    a.R = c->R;
    a.dth = (T)(dt / c->h);
    a.dh = (T)(dt * c->kappa_h / (c->h * c->h));
    a.advection = (c->flags & WX_ADVECTION) ? 1 : 0;
    a.flag_idx = c->flag_idx;
    a.side = c->flag_side;
    a.n_list = c->n_list;
    a.Uw0 = (const T *)c->Uw0;
    a.Vs0 = (const T *)c->Vs0;
    a.out_n = (long long)(2 * c->field_cells);
    M.tile0 = tile0;
    M.gx = (c->nx + kTileX - 1) / kTileX;
    M.gy = (c->ny + ty - 1) / ty;
}

template <typename T, int TY, int KB, int KMODE, bool PHYS, bool SUMS, bool TMF, bool RKB = false>
static int launch_batch_t(wx_ctx *const *mem, int n, const StepCfg &cfg, int num_sms, unsigned *status,
                          cudaStream_t s, std::string &err) {
    auto kern = step_kernel<T, TY, KB, KMODE, PHYS, SUMS, TMF, RKB>;
    Members<T> ms;
    long total = 0;
    int nz_max = 1;
    // the work list takes the largest members (cells) first and the smallest
    // last (measured on the 16-member ensemble: 0.767 ms per step, against
    // 0.789 ms with the deepest members first and 0.800 ms in the given
    // order)
    int ord[kMaxMembers];
    for (int i = 0; i < n; ++i) ord[i] = i;
    std::stable_sort(ord, ord + n, [&](int x, int y) {
        return (long)mem[x]->nx * mem[x]->ny * mem[x]->nz > (long)mem[y]->nx * mem[y]->ny * mem[y]->nz;
    });
    for (int k = 0; k < n; ++k) {
        const int i = ord[k];
        fill_member<T>(mem[i], ms.m[k], total, TY);
        total += (long)ms.m[k].gx * ms.m[k].gy;
        nz_max = std::max(nz_max, mem[i]->nz);
    }
    ms.n = n;
    ms.nz_max = nz_max;
    ms.total = total;
    ms.status = status;
    // an RK3 stage's slots also hold the base boxes: as many as fit
    int stages = cfg.stages;
    while (RKB && stages > 2 && plan_smem(nz_max, TY, stages, KB, (int)sizeof(T), false, TMF, true).total > 227 * 1024)
        --stages;
    const SmemPlan pl = plan_smem(nz_max, TY, stages, KB, (int)sizeof(T), KMODE == 1, TMF, RKB);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, pl.total);
    if (e != cudaSuccess) {
        err = std::string("smem attr: ") + cudaGetErrorString(e);
        return WX_ECUDA;
    }
    // persistent CTAs: no more than fit on the SMs at once (registers,
    // shared memory, TMEM columns)
    int fit = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, kern, 32 * (TY + 1), pl.total);
    if (e != cudaSuccess || fit < 1) {
        err = std::string("step kernel occupancy: ") + (e != cudaSuccess ? cudaGetErrorString(e) : "no CTA fits");
        return WX_ECUDA;
    }
    if (TMF) fit = std::min(fit, 512 / (int)kTmemCols(TY));
    const long resident = (long)num_sms * std::min(cfg.ctas_per_sm, fit);
    dim3 grid((unsigned)std::max(1L, std::min(total, resident)));
    dim3 block(32, TY + 1);
    kern<<<grid, block, pl.total, s>>>(ms, stages, cfg.prefetch);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        err = std::string("step kernel: ") + cudaGetErrorString(e);
        return WX_ECUDA;
    }
    return WX_OK;
}

template <typename T, int KMODE, bool PHYS, bool SUMS>
static int dispatch_ty(wx_ctx *const *mem, int n, const StepCfg &cfg, int sms, unsigned *st, cudaStream_t s,
                       std::string &err) {
    int nz_max = 1;
    for (int i = 0; i < n; ++i) nz_max = std::max(nz_max, mem[i]->nz);
    if constexpr (std::is_same<T, float>::value && KMODE != 1) {
        if (tmem_nz(4, nz_max, false) && tmem_shape(cfg.ty, cfg.kb)) {
            if constexpr (!SUMS)
                if (mem[0]->stage_base >= 0)  // an RK3 stage writing phi^n + (E - phi_s)
                    return launch_batch_t<T, 12, 4, KMODE, PHYS, SUMS, true, true>(mem, n, cfg, sms, st, s, err);
            return launch_batch_t<T, 12, 4, KMODE, PHYS, SUMS, true>(mem, n, cfg, sms, st, s, err);
        }
    }
    if (mem[0]->stage_base >= 0) {
        err = "RK3 stage launches with a base state need the TMEM variant";
        return WX_EUNSUPPORTED;
    }
    switch (cfg.ty * 10 + cfg.kb) {
        case 12: return launch_batch_t<T, 1, 2, KMODE, PHYS, SUMS, false>(mem, n, cfg, sms, st, s, err);
        case 22: return launch_batch_t<T, 2, 2, KMODE, PHYS, SUMS, false>(mem, n, cfg, sms, st, s, err);
        case 42: return launch_batch_t<T, 4, 2, KMODE, PHYS, SUMS, false>(mem, n, cfg, sms, st, s, err);
        case 82: return launch_batch_t<T, 8, 2, KMODE, PHYS, SUMS, false>(mem, n, cfg, sms, st, s, err);
        case 24: return launch_batch_t<T, 2, 4, KMODE, PHYS, SUMS, false>(mem, n, cfg, sms, st, s, err);
        case 44: return launch_batch_t<T, 4, 4, KMODE, PHYS, SUMS, false>(mem, n, cfg, sms, st, s, err);
        case 84: return launch_batch_t<T, 8, 4, KMODE, PHYS, SUMS, false>(mem, n, cfg, sms, st, s, err);
        default: err = "unsupported tile rows / planes per stage"; return WX_EUNSUPPORTED;
    }
}

template <typename T, int KMODE>
static int dispatch_flags(wx_ctx *const *mem, int n, const StepCfg &cfg, int sms, unsigned *st, cudaStream_t s,
                          std::string &err) {
    const unsigned f = mem[0]->flags;
    const bool phys = f & WX_PHYSICS, sums = f & WX_SUMS;
    if (phys && sums) return dispatch_ty<T, KMODE, true, true>(mem, n, cfg, sms, st, s, err);
    if (phys) return dispatch_ty<T, KMODE, true, false>(mem, n, cfg, sms, st, s, err);
    if (sums) return dispatch_ty<T, KMODE, false, true>(mem, n, cfg, sms, st, s, err);
    return dispatch_ty<T, KMODE, false, false>(mem, n, cfg, sms, st, s, err);
}

template <typename T>
static int dispatch_kmode(wx_ctx *const *mem, int n, const StepCfg &cfg, int sms, unsigned *st, cudaStream_t s,
                          std::string &err) {
    // members share kappa_mult use; one with listed columns takes the whole
    // batch through the listing variant (members without any list none)
    if constexpr (std::is_same<T, float>::value) {
        bool any = false;
        for (int i = 0; i < n; ++i) any = any || mixed(mem[i]);
        if (any) return dispatch_flags<T, 2>(mem, n, cfg, sms, st, s, err);
    }
    if (!per_col(mem[0])) return dispatch_flags<T, 0>(mem, n, cfg, sms, st, s, err);
    if constexpr (std::is_same<T, double>::value) return dispatch_flags<T, 1>(mem, n, cfg, sms, st, s, err);
    err = "per-column elimination is built for FP64 storage only";
    return WX_EUNSUPPORTED;
}

// The per-member kernels that follow the step kernel: the side solve of
// WX_MIXED and the sums reduction; then the member's buffers swap.
static int after_step(wx_ctx *c, int ty_used, cudaStream_t s, long *launches) {
    const int dst = 1 - c->cur;
    const bool sums = c->flags & WX_SUMS;
    if (mixed(c) && (c->flags & WX_PHYSICS)) {
        const int rc = launch_mixed_fixup(c, dst, sums, s);
        if (rc != WX_OK) return rc;
        ++*launches;
    }
    if (sums) {
        const long ntiles = (long)((c->nx + kTileX - 1) / kTileX) * ((c->ny + ty_used - 1) / ty_used);
        const long ncorr = (mixed(c) && (c->flags & WX_PHYSICS)) ? c->n_list : 0;
        sums_finalize<<<kFinBlocks, 256, 0, s>>>(c->partials, ntiles, c->flag_corr, ncorr, c->h * c->h,
                                                 c->fin_park, c->fin_ticket, c->sums_ring, c->d_sums_count,
                                                 c->sums_cap);
        WX_CK(cudaGetLastError(), "sums kernel");
        ++*launches;
    }
    if (c->stage_in < 0) c->cur = dst;  // an RK3 stage leaves the buffer order to its driver
    return WX_OK;
}

int launch_batch(wx_ctx *const *mem, int n, const StepCfg &cfg, unsigned *status, cudaStream_t s,
                 long *launches, std::string &err) {
    if (n < 1 || n > kMaxMembers) {
        err = "batch size out of range";
        return WX_EINVAL;
    }
    const int sms = mem[0]->num_sms;
    const int rc = (mem[0]->t_bytes == 4) ? dispatch_kmode<float>(mem, n, cfg, sms, status, s, err)
                                          : dispatch_kmode<double>(mem, n, cfg, sms, status, s, err);
    if (rc != WX_OK) return rc;
    ++*launches;
    for (int i = 0; i < n; ++i) {
        const int r2 = after_step(mem[i], cfg.ty, s, launches);
        if (r2 != WX_OK) {
            err = mem[i]->err;
            return r2;
        }
    }
    return WX_OK;
}

int launch_step(wx_ctx *c, cudaStream_t s, long *launches) {
    wx_ctx *mem[1] = {c};
    return launch_batch(mem, 1, c->cfg, c->d_status, s, launches, c->err);
}

// ------------------------------------------------------------- WX_RK3
// phi_out = phi_n + (E - phi_s) over whole state buffers (both fields,
// ghost ring and padding included): E = phi_s + c dt L(phi_s) is what the
// step kernel writes for one stage, so this is phi_n + c dt L(phi_s).
template <typename T>
__global__ void rk_combine_kernel(const T *__restrict__ base, const T *E, const T *S, T *out, size_t n) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        out[e] = base[e] + (E[e] - S[e]);
}

// The last RK3 stage's combine fused with the column physics, one thread
// per column: phi3 = A + (E - S) for T and q (out holds E, the stage
// kernel's output), q^{n+1} = q3, and T^{n+1} = the column physics of
// (T3, q3), all written over `out` with the ghost copies.  Without a
// per-column kappa_mult the elimination comes from the table, run from the
// top with the heating folded into the back substitution as in the step
// kernel (FMA-only recurrences; scratch F_k in shared memory); with one,
// the forward sweep divides per level (scratch c'_k, d'_k).
template <typename T, bool TABLE>
__global__ void __launch_bounds__(64) rk_physics_kernel(T *__restrict__ out, const T *__restrict__ A,
                                                        const T *__restrict__ S, int nx, int ny, int nz, int P,
                                                        int R, const T *__restrict__ km,
                                                        const Q4<T> *__restrict__ tab,
                                                        unsigned *__restrict__ status) {
    extern __shared__ __align__(16) unsigned char psm[];
    T *scr = reinterpret_cast<T *>(psm);  // [level][thread], 1 or 2 arrays
    const int t = threadIdx.x, nt = blockDim.x;
    const long c = (long)blockIdx.x * nt + t;
    if (c >= (long)nx * ny) return;
    const int j = (int)(c / nx), i = (int)(c - (long)j * nx);
    const size_t plane = (size_t)R * P, off = (size_t)(j + 1) * P + i + kGhostX;
    auto at = [&](int k, int f) { return off + (size_t)(2 * k + f) * plane; };
    auto phi3 = [&](int k, int f) { const size_t o = at(k, f); return A[o] + (out[o] - S[o]); };
    auto put = [&](int k, int f, T v) {
        T *row = out + at(k, f);
        row[0] = v;
        if (i == 0) row[nx] = v;                   // -> right ghost column
        if (i == nx - 1) row[-nx] = v;             // -> left ghost column
        if (j == 0) row[(size_t)ny * P] = v;       // -> top ghost row
        if (j == ny - 1) row[-(long)ny * P] = v;   // -> bottom ghost row
    };
    const Q4<T> *tB = tab + REC_B * nz, *tC = tab + REC_C * nz, *tD = tab + REC_D * nz, *tE = tab + REC_E * nz;
    bool ok = true;
    if (TABLE) {
        // pass 1, top down: q3 stored, optical depth, elimination, F_{k+1}
        T tau = 0, Etop = 1, f_up = 0, h_up = 0;
        for (int k = nz - 1; k >= 0; --k) {
            const T q3 = phi3(k, 1), t3 = phi3(k, 0);
            put(k, 1, q3);
            ok = ok && isfinite((double)q3);
            const T taub = tau + tB[k].z * q3;
            const T Eb = exp2_neg(taub);
            const T h = tC[k].x * (Etop - Eb);
            const T f = (t3 + tC[k].z * f_up) * tD[k].x;
            if (k < nz - 1) scr[(size_t)(k + 1) * nt + t] = f_up + h_up + tD[k + 1].z * h;
            f_up = f;
            h_up = h;
            Etop = Eb;
            tau = taub;
        }
        scr[t] = f_up + h_up;  // level 0: e_0 = 0
        // pass 2, bottom up: T_k = F_k - e_k T_{k-1}
        T prev = 0;
        for (int k = 0; k < nz; ++k) {
            const T v = scr[(size_t)k * nt + t] - tD[k].z * prev;
            ok = ok && isfinite((double)v);
            put(k, 0, v);
            prev = v;
        }
    } else {
        T *cp = scr, *dp = scr + (size_t)nz * nt;
        const T s = km[c];
        ThomasSweep<T> fw;
        for (int k = 0; k < nz; ++k) {
            cp[(size_t)k * nt + t] = fw.level(-s * tE[k].x, -s * tE[k].y, phi3(k, 0));
            dp[(size_t)k * nt + t] = fw.d;
        }
        T x = 0, tau = 0, Etop = 1;
        for (int k = nz - 1; k >= 0; --k) {
            const T q3 = phi3(k, 1);
            x = dp[(size_t)k * nt + t] - cp[(size_t)k * nt + t] * x;
            const T taub = tau + tB[k].z * q3;
            const T Eb = exp2_neg(taub);
            const T v = x + tC[k].x * (Etop - Eb);
            ok = ok && isfinite((double)v) && isfinite((double)q3);
            put(k, 0, v);
            put(k, 1, q3);
            Etop = Eb;
            tau = taub;
        }
    }
    if (!ok) atomicOr(status, ST_NONFINITE);
}

// One RK3 step: with A = the current state, B = the other ping-pong buffer
// and C = the stage buffer,
//   stage 1: B <- step_{dt/3}(A)              (phi1 = A + dt/3 L(A))
//   stage 2: C <- step_{dt/2}(B); C <- A + (C - B)
//   stage 3: B <- step_{dt}(C);   then, fused with the column physics,
//            phi3 = A + (B - C) and B <- physics(phi3)  (WX_PHYSICS), or
//            B <- A + (B - C)
//   B becomes current.  The step kernel runs without physics in every stage.
template <typename T> static int rk_combine(wx_ctx *c, int base, int e, int st, int out, cudaStream_t s) {
    const size_t n = 2 * c->field_cells;
    rk_combine_kernel<T><<<grid_for(n), 256, 0, s>>>((const T *)c->fld[base], (const T *)c->fld[e],
                                                     (const T *)c->fld[st], (T *)c->fld[out], n);
    WX_CK(cudaGetLastError(), "RK3 combine kernel");
    return WX_OK;
}

template <typename T> static int rk_physics(wx_ctx *c, int A, int B, int C, cudaStream_t s) {
    constexpr int nt = 64;
    const bool table = c->kmult == nullptr;
    const size_t sm = (size_t)nt * c->nz * sizeof(T) * (table ? 1 : 2);
    const unsigned g = (unsigned)(((long)c->nx * c->ny + nt - 1) / nt);
    auto kern = table ? rk_physics_kernel<T, true> : rk_physics_kernel<T, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess) {
        kern<<<g, nt, sm, s>>>((T *)c->fld[B], (const T *)c->fld[A], (const T *)c->fld[C], c->nx, c->ny, c->nz,
                               c->P, c->R, (const T *)c->kmult, (const Q4<T> *)c->tab, c->d_status);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "RK3 physics kernel");
    return WX_OK;
}

// RK3 on the TMEM variant: three stage launches of the step kernel, each
// writing its stage's state itself (the base state phi^n rides in the same
// TMA ring as the stage input), the last fused with the column physics:
//   stage 1: B <- step_{dt/3}(A)                     (phi1)
//   stage 2: C <- A + (step_{dt/2}(B) - B)           (phi2)
//   stage 3: B <- physics(A + (step_{dt}(C) - C))    (q^{n+1} = q3)
// followed by the side solve of listed columns.  Per cell and step: 16 B,
// then 24 B twice (read phi_s and phi^n, write), 64 B in all.
static int launch_rk3_fused(wx_ctx *c, cudaStream_t s, long *launches) {
    const int A = c->cur, B = 1 - c->cur, C = 2;
    const size_t tbytes = (size_t)c->nz * kTabRec * 4 * c->t_bytes;
    int rc = encode_tmap_interior(c, A, c->cfg.ty, c->cfg.kb, &c->tmap_rkbase);
    if (rc != WX_OK) return rc;
    const unsigned saved = c->flags;
    const int in[3] = {A, B, C}, out[3] = {B, C, B};
    const double dts[3] = {c->dt / 3.0, c->dt / 2.0, c->dt};
    for (int st = 0; st < 3 && rc == WX_OK; ++st) {
        c->stage_in = in[st];
        c->stage_out = out[st];
        c->stage_dt = dts[st];
        c->stage_tab = (const char *)c->tab_rk + st * tbytes;
        c->stage_base = st == 0 ? -1 : A;
        c->flags = st == 2 ? saved : (saved & WX_ADVECTION);
        rc = launch_step(c, s, launches);
    }
    c->stage_in = c->stage_out = c->stage_base = -1;
    c->stage_tab = nullptr;
    c->flags = saved;
    if (rc != WX_OK) return rc;
    c->cur = B;
    return WX_OK;
}

int launch_rk3_step(wx_ctx *c, cudaStream_t s, long *launches) {
    if (use_tmem(c, c->cfg)) return launch_rk3_fused(c, s, launches);
    const int A = c->cur, B = 1 - c->cur, C = 2;
    const size_t tbytes = (size_t)c->nz * kTabRec * 4 * c->t_bytes;
    const unsigned saved = c->flags;
    const bool f32 = c->t_bytes == 4;
    c->flags = saved & WX_ADVECTION;
    int rc = WX_OK;
    const int in[3] = {A, B, C}, out[3] = {B, C, B};
    const double dts[3] = {c->dt / 3.0, c->dt / 2.0, c->dt};
    for (int st = 0; st < 3 && rc == WX_OK; ++st) {
        c->stage_in = in[st];
        c->stage_out = out[st];
        c->stage_dt = dts[st];
        c->stage_tab = (const char *)c->tab_rk + st * tbytes;
        rc = launch_step(c, s, launches);
        if (rc == WX_OK && (st == 1 || (st == 2 && !(saved & WX_PHYSICS)))) {
            rc = f32 ? rk_combine<float>(c, A, out[st], in[st], out[st], s)
                     : rk_combine<double>(c, A, out[st], in[st], out[st], s);
            ++*launches;
        }
    }
    c->stage_in = c->stage_out = -1;
    c->stage_tab = nullptr;
    c->flags = saved;
    if (rc != WX_OK) return rc;
    if (saved & WX_PHYSICS) {
        const int r2 = f32 ? rk_physics<float>(c, A, B, C, s) : rk_physics<double>(c, A, B, C, s);
        if (r2 != WX_OK) return r2;
        ++*launches;
    }
    c->cur = B;
    return WX_OK;
}

}  // namespace wx
