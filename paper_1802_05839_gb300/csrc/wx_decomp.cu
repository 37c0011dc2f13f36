// wx_decomp.cu -- horizontal (IJ) block decomposition of one periodic grid
// with a depth-1 halo exchange: the paper's multi-GPU layout of ASUCA (App.
// F decomposition table; Sec. 5.4, where the exchange is the communication
// share of the strong-scaling runs), run as simulated ranks on one GPU.
//
// Every block is an ordinary context whose west-face / south-face winds of
// the first column / row come from its neighbours.  A step is one launch of
// the step kernel over all blocks' tiles (each block's own periodic ghost
// copies are made and then overwritten), then one launch of the exchange
// kernel, which copies each block's four edge lines (both fields, every
// level) into its neighbours' ghost lines; it also runs after a load.
// Corners are not exchanged: neither the 7-point diffusion nor the upwind
// fluxes read them.  Because every interior cell sees the same
// neighbour values, winds, coefficients and tables as in the undecomposed
// grid, and its arithmetic does not depend on where its tile starts, the
// blocks' interiors equal the undecomposed step bit for bit.
#include <algorithm>
#include <cstring>
#include <new>

#include "wx_internal.cuh"

using namespace wx;

namespace {

// One ghost strip of one block for a buffer parity: `n` cells per (k, f)
// plane, read from src[src_off + p*src_plane + i*src_step] and written to
// dst[dst_off + p*dst_plane + i*dst_step] for plane p and cell i.
struct Strip {
    const void *src;  // the source block's state buffer
    void *dst;        // the receiving block's state buffer
    long src_off, dst_off;  // first cell of the line in plane 0 (elements)
    long src_plane, dst_plane;
    long long src_n, dst_n;  // elements of each buffer
    int n, src_step, dst_step, pad;
};

// One cell per thread (blockIdx.x = strip, blockIdx.y * 256 + thread = cell
// of the strip's n x nplanes), so that every copy's load is in flight at
// once: the column strips are one element per 32-byte sector and the kernel
// is latency bound.
template <typename T>
__global__ void __launch_bounds__(256) halo_exchange_kernel(const Strip *__restrict__ strips, int nplanes,
                                                            unsigned *__restrict__ status) {
    const Strip s = strips[blockIdx.x];
    const T *__restrict__ src = static_cast<const T *>(s.src);
    T *__restrict__ dst = static_cast<T *>(s.dst);
    const unsigned total = (unsigned)s.n * (unsigned)nplanes;
    for (unsigned e = blockIdx.y * blockDim.x + threadIdx.x; e < total; e += gridDim.y * blockDim.x) {
        const unsigned p = e / (unsigned)s.n, i = e - p * (unsigned)s.n;
        const long so = s.src_off + (long)p * s.src_plane + (long)i * s.src_step;
        const long d = s.dst_off + (long)p * s.dst_plane + (long)i * s.dst_step;
        if (WX_IN(so, s.src_n, status) && WX_IN(d, s.dst_n, status)) dst[d] = src[so];
    }
}

thread_local std::string g_dom_create_error;

bool split_ok(const int *sp, int parts, int n) {
    if (sp[0] != 0 || sp[parts] != n) return false;
    for (int i = 0; i < parts; ++i)
        if (sp[i + 1] <= sp[i]) return false;
    return true;
}

// Block boundaries: the caller's, or the even split floor(i n / parts).
bool make_split(const int *given, int parts, int n, std::vector<int> &out) {
    out.resize(parts + 1);
    if (given)
        std::copy(given, given + parts + 1, out.begin());
    else
        for (int i = 0; i <= parts; ++i) out[i] = (int)((long)i * n / parts);
    return split_ok(out.data(), parts, n);
}

void plan_of(const std::vector<int> &xs, const std::vector<int> &ys, int r, wx_halo_strip out[4]) {
    const int px = (int)xs.size() - 1, py = (int)ys.size() - 1;
    const int ix = r % px, iy = r / px;
    const int iw = (ix + px - 1) % px, ie = (ix + 1) % px, is = (iy + py - 1) % py, in = (iy + 1) % py;
    const int nxr = xs[ix + 1] - xs[ix], nyr = ys[iy + 1] - ys[iy];
    const int nxw = xs[iw + 1] - xs[iw], nys = ys[is + 1] - ys[is];
    out[0] = {WX_HALO_WEST, iy * px + iw, nxw - 1, -1, nyr};
    out[1] = {WX_HALO_EAST, iy * px + ie, 0, nxr, nyr};
    out[2] = {WX_HALO_SOUTH, is * px + ix, nys - 1, -1, nxr};
    out[3] = {WX_HALO_NORTH, in * px + ix, 0, nyr, nxr};
}

}  // namespace

struct wx_dom {
    int nx = 0, ny = 0, nz = 0, dtype = 0, px = 0, py = 0;
    std::vector<int> xs, ys;
    std::vector<wx_ctx *> blk;
    StepCfg cfg;
    unsigned *d_status = nullptr;
    Strip *d_strips = nullptr;  // [2 parities][4 * blocks]
    bool loaded = false;
    cudaStream_t last_stream = nullptr;
    long last_launches = 0;
    std::string err;
};

static int dfail(wx_dom *d, int code, const std::string &m) {
    if (d)
        d->err = m;
    else
        g_dom_create_error = m;
    return code;
}

extern "C" int wx_dom_halo_plan(int nx, int ny, int px, int py, const int *xsplit, const int *ysplit, int r,
                                wx_halo_strip out[4]) {
    if (!out || nx < 1 || ny < 1 || px < 1 || py < 1 || px > nx || py > ny || r < 0 || r >= px * py)
        return WX_EINVAL;
    std::vector<int> xs, ys;
    if (!make_split(xsplit, px, nx, xs) || !make_split(ysplit, py, ny, ys)) return WX_EINVAL;
    plan_of(xs, ys, r, out);
    return WX_OK;
}

// Device strips of both buffer parities, from the host plan.  Cell (i, j)
// of a block sits at row jp = j + 1, column ip = i + kGhostX of each plane.
static int build_strips(wx_dom *d) {
    const int R = (int)d->blk.size();
    std::vector<Strip> h(2 * 4 * (size_t)R);
    for (int par = 0; par < 2; ++par)
        for (int r = 0; r < R; ++r) {
            wx_halo_strip pl[4];
            plan_of(d->xs, d->ys, r, pl);
            const wx_ctx *dc = d->blk[r];
            for (int s = 0; s < 4; ++s) {
                const wx_ctx *sc = d->blk[pl[s].src];
                const bool col = pl[s].dir == WX_HALO_WEST || pl[s].dir == WX_HALO_EAST;
                // first cell of the line in plane 0, in elements
                const long soff = col ? (long)1 * sc->P + kGhostX + pl[s].src_line
                                      : (long)(pl[s].src_line + 1) * sc->P + kGhostX;
                const long doff = col ? (long)1 * dc->P + kGhostX + pl[s].dst_line
                                      : (long)(pl[s].dst_line + 1) * dc->P + kGhostX;
                Strip &st = h[((size_t)par * R + r) * 4 + s];
                st.src = sc->fld[par];
                st.dst = dc->fld[par];
                st.src_off = soff;
                st.dst_off = doff;
                st.src_plane = (long)sc->plane_cells;
                st.dst_plane = (long)dc->plane_cells;
                st.src_n = (long long)(2 * sc->field_cells);
                st.dst_n = (long long)(2 * dc->field_cells);
                st.n = pl[s].len;
                st.src_step = col ? sc->P : 1;
                st.dst_step = col ? dc->P : 1;
                st.pad = 0;
            }
        }
    if (cudaMalloc(&d->d_strips, h.size() * sizeof(Strip)) != cudaSuccess) {
        cudaGetLastError();
        d->d_strips = nullptr;
        return dfail(d, WX_ENOMEM, "wx_dom: strip list allocation failed");
    }
    if (cudaMemcpy(d->d_strips, h.data(), h.size() * sizeof(Strip), cudaMemcpyHostToDevice) != cudaSuccess)
        return dfail(d, WX_ECUDA, "wx_dom: strip list upload failed");
    return WX_OK;
}

static int launch_exchange(wx_dom *d, cudaStream_t s) {
    const int R = (int)d->blk.size(), par = d->blk[0]->cur;
    const int nplanes = 2 * d->nz;
    long maxn = 1;
    for (int r = 0; r < R; ++r) maxn = std::max<long>(maxn, std::max(d->blk[r]->nx, d->blk[r]->ny));
    if (maxn * nplanes >= (1L << 32) - 65536L * 256)
        return dfail(d, WX_EUNSUPPORTED, "halo exchange: a strip holds 2^32 cells or more");
    const long per = (maxn * nplanes + 255) / 256;
    dim3 grid((unsigned)(4 * R), (unsigned)std::min<long>(per, 65535));
    const Strip *st = d->d_strips + (size_t)par * 4 * R;
    if (d->blk[0]->t_bytes == 4)
        halo_exchange_kernel<float><<<grid, 256, 0, s>>>(st, nplanes, d->d_status);
    else
        halo_exchange_kernel<double><<<grid, 256, 0, s>>>(st, nplanes, d->d_status);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return dfail(d, WX_ECUDA, std::string("halo exchange kernel: ") + cudaGetErrorString(e));
    return WX_OK;
}

extern "C" int wx_dom_create(int nx, int ny, int nz, int dtype, int px, int py, const int *xsplit,
                             const int *ysplit, wx_dom **out) {
    if (!out) return dfail(nullptr, WX_EINVAL, "wx_dom_create: out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || px < 1 || py < 1)
        return dfail(nullptr, WX_EINVAL, "wx_dom_create: sizes and block counts must be >= 1");
    if ((long)px * py > kMaxMembers) return dfail(nullptr, WX_EUNSUPPORTED, "wx_dom_create: at most 16 blocks");
    if (px > nx || py > ny) return dfail(nullptr, WX_EINVAL, "wx_dom_create: more blocks than columns or rows");
    wx_dom *d = new (std::nothrow) wx_dom();
    if (!d) return dfail(nullptr, WX_ENOMEM, "wx_dom_create: host allocation failed");
    d->nx = nx;
    d->ny = ny;
    d->nz = nz;
    d->dtype = dtype;
    d->px = px;
    d->py = py;
    auto bail = [&](int code) {
        g_dom_create_error = d->err;
        wx_dom_destroy(d);
        return code;
    };
    if (!make_split(xsplit, px, nx, d->xs) || !make_split(ysplit, py, ny, d->ys)) {
        d->err = "wx_dom_create: splits must run 0 = s_0 < s_1 < ... < s_parts = n";
        return bail(WX_EINVAL);
    }
    for (int iy = 0; iy < py; ++iy)
        for (int ix = 0; ix < px; ++ix) {
            const int nxr = d->xs[ix + 1] - d->xs[ix], nyr = d->ys[iy + 1] - d->ys[iy];
            wx_ctx *c = nullptr;
            const int rc = wx_create(nxr, nyr, nz, dtype, &c);
            if (rc != WX_OK) {
                d->err = std::string("block ") + std::to_string(d->blk.size()) + ": " + wx_last_error(nullptr);
                return bail(rc);
            }
            d->blk.push_back(c);
            if (cudaMalloc(&c->Uw0, (size_t)nyr * c->t_bytes) != cudaSuccess ||
                cudaMalloc(&c->Vs0, (size_t)nxr * c->t_bytes) != cudaSuccess ||
                cudaMemset(c->Uw0, 0, (size_t)nyr * c->t_bytes) != cudaSuccess ||
                cudaMemset(c->Vs0, 0, (size_t)nxr * c->t_bytes) != cudaSuccess) {
                cudaGetLastError();
                d->err = "wx_dom_create: halo wind allocation failed";
                return bail(WX_ENOMEM);
            }
            c->Uw0_h.assign(nyr, 0.0);
            c->Vs0_h.assign(nxr, 0.0);
        }
    if (cudaMalloc(&d->d_status, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(d->d_status, 0, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        d->err = "wx_dom_create: CUDA set-up failed";
        return bail(WX_ECUDA);
    }
    int rc = build_strips(d);
    if (rc != WX_OK) return bail(rc);
    d->cfg = d->blk[0]->cfg;
    *out = d;
    return WX_OK;
}

extern "C" void wx_dom_destroy(wx_dom *d) {
    if (!d) return;
    for (auto *c : d->blk) wx_destroy(c);
    if (d->d_status) cudaFree(d->d_status);
    if (d->d_strips) cudaFree(d->d_strips);
    delete d;
}

extern "C" const char *wx_dom_last_error(const wx_dom *d) { return d ? d->err.c_str() : g_dom_create_error.c_str(); }
extern "C" int wx_dom_size(const wx_dom *d) { return d ? (int)d->blk.size() : 0; }
extern "C" long wx_dom_last_launches(const wx_dom *d) { return d ? d->last_launches : -1; }
extern "C" wx_ctx *wx_dom_block(wx_dom *d, int r) {
    if (!d || r < 0 || r >= (int)d->blk.size()) return nullptr;
    return d->blk[r];
}

// One launch configuration for every block: the first block's (all blocks
// share nz, dtype and kappa_mult use, so its shared-memory plan is theirs).
static int dom_sync_cfg(wx_dom *d) {
    d->cfg = d->blk[0]->cfg;
    for (auto *c : d->blk)
        if (c->cfg.ty != d->cfg.ty || c->cfg.kb != d->cfg.kb || c->cfg.stages != d->cfg.stages ||
            c->cfg.ctas_per_sm != d->cfg.ctas_per_sm) {
            const int rc = apply_cfg(c, d->cfg);
            if (rc != WX_OK) return dfail(d, rc, c->err);
        }
    return WX_OK;
}

extern "C" int wx_dom_set_params(wx_dom *d, const wx_params *p) {
    if (!d) return WX_EINVAL;
    if (!p) return dfail(d, WX_EINVAL, "wx_dom_set_params: params is NULL");
    if (p->flags & (WX_RK3 | WX_SURROGATE))
        return dfail(d, WX_EUNSUPPORTED, "wx_dom_set_params: WX_RK3 and WX_SURROGATE are not decomposed");
    std::vector<double> km;
    for (size_t r = 0; r < d->blk.size(); ++r) {
        wx_ctx *c = d->blk[r];
        wx_params q = *p;
        if (p->kappa_mult) {
            const int x0 = d->xs[r % d->px], y0 = d->ys[r / d->px];
            km.resize((size_t)c->nx * c->ny);
            for (int j = 0; j < c->ny; ++j)
                std::memcpy(&km[(size_t)j * c->nx], p->kappa_mult + (size_t)(y0 + j) * d->nx + x0,
                            c->nx * sizeof(double));
            q.kappa_mult = km.data();
        }
        const int rc = wx_set_params(c, &q);
        if (rc != WX_OK) return dfail(d, rc, "block " + std::to_string(r) + ": " + c->err);
    }
    return dom_sync_cfg(d);
}

extern "C" int wx_dom_load_fields(wx_dom *d, const double *T, const double *q, const double *U, const double *V) {
    if (!d) return WX_EINVAL;
    if (!T || !q || !U || !V) return dfail(d, WX_EINVAL, "wx_dom_load_fields: NULL array");
    const int nx = d->nx, ny = d->ny, nz = d->nz;
    std::vector<double> Tb, qb, Ub, Vb;
    d->loaded = false;
    for (size_t r = 0; r < d->blk.size(); ++r) {
        wx_ctx *c = d->blk[r];
        const int x0 = d->xs[r % d->px], y0 = d->ys[r / d->px], bx = c->nx, by = c->ny;
        Tb.resize((size_t)nz * by * bx);
        qb.resize(Tb.size());
        Ub.resize((size_t)by * bx);
        Vb.resize(Ub.size());
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < by; ++j) {
                const size_t g = ((size_t)k * ny + y0 + j) * nx + x0, l = ((size_t)k * by + j) * bx;
                std::memcpy(&Tb[l], T + g, bx * sizeof(double));
                std::memcpy(&qb[l], q + g, bx * sizeof(double));
            }
        for (int j = 0; j < by; ++j) {
            std::memcpy(&Ub[(size_t)j * bx], U + (size_t)(y0 + j) * nx + x0, bx * sizeof(double));
            std::memcpy(&Vb[(size_t)j * bx], V + (size_t)(y0 + j) * nx + x0, bx * sizeof(double));
        }
        int rc = wx_load_fields(c, Tb.data(), qb.data(), Ub.data(), Vb.data(), 0);
        if (rc != WX_OK) return dfail(d, rc, "block " + std::to_string(r) + ": " + c->err);
        // the neighbours' face winds west of column 0 and south of row 0
        const int xw = (x0 + nx - 1) % nx, ys = (y0 + ny - 1) % ny;
        for (int j = 0; j < by; ++j) c->Uw0_h[j] = U[(size_t)(y0 + j) * nx + xw];
        for (int i = 0; i < bx; ++i) c->Vs0_h[i] = V[(size_t)ys * nx + x0 + i];
        for (int w = 0; w < 2; ++w) {
            const std::vector<double> &src = w ? c->Vs0_h : c->Uw0_h;
            void *dst = w ? c->Vs0 : c->Uw0;
            cudaError_t e;
            if (c->t_bytes == 4) {
                std::vector<float> f(src.begin(), src.end());
                e = cudaMemcpy(dst, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice);
            } else {
                e = cudaMemcpy(dst, src.data(), src.size() * sizeof(double), cudaMemcpyHostToDevice);
            }
            if (e != cudaSuccess) return dfail(d, WX_ECUDA, std::string("halo winds: ") + cudaGetErrorString(e));
        }
        c->cfl_ok = false;
        ++c->generation;
    }
    int rc = launch_exchange(d, 0);
    if (rc != WX_OK) return rc;
    if (cudaDeviceSynchronize() != cudaSuccess) return dfail(d, WX_ECUDA, "wx_dom_load_fields: exchange failed");
    d->loaded = true;
    return WX_OK;
}

extern "C" int wx_dom_step(wx_dom *d, int n_steps, void *stream) {
    if (!d) return WX_EINVAL;
    if (n_steps < 0) return dfail(d, WX_EINVAL, "wx_dom_step: n_steps < 0");
    if (!d->loaded) return dfail(d, WX_ESTATE, "wx_dom_step: set params and load fields first");
    for (size_t r = 0; r < d->blk.size(); ++r) {
        wx_ctx *c = d->blk[r];
        if (!c->params_set) return dfail(d, WX_ESTATE, "wx_dom_step: set params first");
        const int rc = check_cfl(c);
        if (rc != WX_OK) return dfail(d, rc, "block " + std::to_string(r) + ": " + c->err);
    }
    int rc = dom_sync_cfg(d);
    if (rc != WX_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    d->last_stream = s;
    // every step: the step kernel over all blocks (with the side solve of
    // listed columns, when there are any), then the exchange of the new
    // states' edge lines
    long launches = 0;
    for (int n = 0; n < n_steps; ++n) {
        rc = launch_batch(d->blk.data(), (int)d->blk.size(), d->cfg, d->d_status, s, &launches, d->err);
        if (rc != WX_OK) return rc;
        rc = launch_exchange(d, s);
        if (rc != WX_OK) return rc;
        ++launches;
    }
    for (auto *c : d->blk) c->last_stream = s;
    d->last_launches = launches;
    return WX_OK;
}

extern "C" int wx_dom_sync(wx_dom *d) {
    if (!d) return WX_EINVAL;
    if (cudaStreamSynchronize(d->last_stream) != cudaSuccess) return dfail(d, WX_ECUDA, "wx_dom_sync");
    unsigned st = 0;
    if (cudaMemcpy(&st, d->d_status, sizeof st, cudaMemcpyDeviceToHost) != cudaSuccess)
        return dfail(d, WX_ECUDA, "wx_dom_sync: status");
    if (st) cudaMemset(d->d_status, 0, sizeof st);
    for (size_t r = 0; r < d->blk.size(); ++r) {
        d->blk[r]->last_stream = d->last_stream;
        const int rc = wx_sync(d->blk[r]);
        if (rc != WX_OK) return dfail(d, rc, "block " + std::to_string(r) + ": " + d->blk[r]->err);
    }
    if (st & ST_TIMEOUT) return dfail(d, WX_ETIMEOUT, "a bounded device wait timed out");
    if (st & ST_BOUNDS) return dfail(d, WX_ECUDA, "the halo exchange skipped an out-of-bounds access");
    return WX_OK;
}

extern "C" int wx_dom_read_fields(wx_dom *d, double *T, double *q) {
    if (!d) return WX_EINVAL;
    if (!d->loaded) return dfail(d, WX_ESTATE, "wx_dom_read_fields: no fields loaded");
    const int nx = d->nx, ny = d->ny, nz = d->nz;
    std::vector<double> Tb, qb;
    for (size_t r = 0; r < d->blk.size(); ++r) {
        wx_ctx *c = d->blk[r];
        const int x0 = d->xs[r % d->px], y0 = d->ys[r / d->px], bx = c->nx, by = c->ny;
        Tb.resize((size_t)nz * by * bx);
        qb.resize(Tb.size());
        const int rc = wx_read_fields(c, T ? Tb.data() : nullptr, q ? qb.data() : nullptr);
        if (rc != WX_OK) return dfail(d, rc, "block " + std::to_string(r) + ": " + c->err);
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < by; ++j) {
                const size_t g = ((size_t)k * ny + y0 + j) * nx + x0, l = ((size_t)k * by + j) * bx;
                if (T) std::memcpy(T + g, &Tb[l], bx * sizeof(double));
                if (q) std::memcpy(q + g, &qb[l], bx * sizeof(double));
            }
    }
    return WX_OK;
}

extern "C" int wx_dom_get_sums(wx_dom *d, double *mass_q, double *energy_T, int max_steps, int *n_out) {
    if (!d) return WX_EINVAL;
    if (max_steps < 0) return dfail(d, WX_EINVAL, "wx_dom_get_sums: max_steps < 0");
    std::vector<double> m(max_steps), e(max_steps);
    int n0 = -1;
    for (size_t r = 0; r < d->blk.size(); ++r) {
        int n = 0;
        const int rc = wx_get_sums(d->blk[r], m.data(), e.data(), max_steps, &n);
        if (rc != WX_OK) return dfail(d, rc, "block " + std::to_string(r) + ": " + d->blk[r]->err);
        if (n0 >= 0 && n != n0) return dfail(d, WX_ESTATE, "wx_dom_get_sums: blocks recorded different step counts");
        if (n0 < 0) {
            n0 = n;
            for (int s = 0; s < n; ++s) {
                if (mass_q) mass_q[s] = 0.0;
                if (energy_T) energy_T[s] = 0.0;
            }
        }
        for (int s = 0; s < n; ++s) {
            if (mass_q) mass_q[s] += m[s];
            if (energy_T) energy_T[s] += e[s];
        }
    }
    if (n_out) *n_out = n0 < 0 ? 0 : n0;
    return WX_OK;
}
