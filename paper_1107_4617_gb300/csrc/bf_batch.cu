// Host side of the batched entry points: builds the tile table of many
// uneven images (each with its own r, N, gamma, a_k) in the caller's
// workspace and launches the persistent tile-queue kernels. Plain sums run on
// the skewed-strip engine (two persistent launches, 128- and 256-thread
// strips); Kahan-compensated sums on the single-pass kernel.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "bf_internal.cuh"
#include "bf_launch.cuh"
#include "bf_trace.cuh"

namespace bf {

// Rows per band in a batch on the skewed-strip engine: tall enough that the
// strip's skew (Wi steps) and the 2r warm-up rows stay a minor cost, small
// enough that the tiles still balance over the SMs (on 256 images of sides
// 64..2048, 1024-row bands ran 9 % faster than 512; the batch autotuner
// refines this per batch).
static int sys_batch_rows(int r, int H, const bf_opts* o) {
    if (o && o->tile_h > 0) return o->tile_h < H ? o->tile_h : H;
    int hb = 1024;
    if (hb < 8 * r) hb = 8 * r;
    return hb < H ? hb : H;
}

// Rows per band for the single-pass kernel (Kahan batches).
static int v0_batch_rows(int r, const bf_opts* o) {
    if (o && o->tile_h > 0) return o->tile_h;
    int hb = 128;
    if (hb < 4 * r) hb = 4 * r;
    return hb;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static size_t v0_table_bytes(int n) {
    return sizeof(BatchTable) + (size_t)(n > 1 ? n - 1 : 0) * sizeof(BatchImage);
}

static size_t sys_table_bytes(int n) {
    return sizeof(SysBatchTable) + (size_t)(n > 1 ? n - 1 : 0) * sizeof(SysBatchImage);
}

// Strip width of an image on the skewed-strip engine (same rule as a single
// image), or 0 when the strip would keep fewer than 16 output columns. The
// persistent launches run 128- or 256-thread CTAs, so a batch takes only
// those two widths.
static int sys_width(int r, const bf_opts* o) {
    int wi = (r <= 40) ? 128 : 256;
    if (o && o->tile_w > 0) {
        if (o->tile_w != 128 && o->tile_w != 256) return 0;
        wi = o->tile_w;
    }
    if (wi % 32 != 0 || wi > SYS_MAX_THREADS || wi - 2 * r < 16) return 0;
    return wi;
}

struct Plan {
    FwdParams p;
    int wi, gx, gy, Hb, nch;
    int group;  // persistent launch (SysBatchTable::g)
    int kind;   // its specialised kernel within the group, or -1
    long long cost;
};

static bf_status plan_image(const bf_desc& d, const bf_opts* opts, Plan* pl) {
    bf_opts o;
    if (opts) o = *opts; else bf_default_opts(&o);
    o.tile_w = 0;
    o.tile_h = 0;
    o.save_for_backward = 0;
    int nt = 0, gx = 0, gy = 0;
    bf_status st = fill_fwd_params(d.img, d.out, nullptr, d.H, d.W, d.pitch, d.r, d.sigma_r, d.T,
                                   d.N, &o, &pl->p, &nt, &gx, &gy);
    if (st != BF_OK) return st;
    pl->p.den = d.den;
    if (d.den && (d.den == d.out || (const void*)d.den == d.img)) return BF_ERR_INVALID_ARG;
    pl->wi = sys_width(d.r, opts);
    if (!pl->wi) return BF_ERR_UNSUPPORTED;
    // the engine addresses one image with 32-bit element offsets
    if ((long long)(d.H + 2 * pl->wi + 4 * d.r) * pl->p.ld >= 0x7fffffffLL) return BF_ERR_UNSUPPORTED;
    const int Tw = pl->wi - 2 * d.r;
    pl->Hb = sys_batch_rows(d.r, d.H, opts);
    pl->gx = (d.W + Tw - 1) / Tw;
    pl->gy = (d.H + pl->Hb - 1) / pl->Hb;
    pl->nch = sys_chunks(pl->p.K, false, 0);
    if (pl->nch > SYS_BATCH_MAX_CHUNKS) return BF_ERR_UNSUPPORTED;
    int kg = 1;
    pl->kind = (pl->wi <= 128 && pl->nch == 1) ? sys_batch_kind(pl->p.K, pl->p.kstart, &kg) : -1;
    pl->group = pl->wi > 128 ? 2 : (pl->kind >= 0 ? kg : 1);
    pl->cost = (long long)(pl->Hb + 2 * d.r + pl->wi) * (pl->p.K + 2);
    return BF_OK;
}

// Workspace: table, then one H x W den accumulator per image whose harmonics
// run in two chunks.
static bf_status sys_layout(const bf_desc* descs, int n, const bf_opts* opts,
                            std::vector<Plan>* plans, size_t* total) {
    plans->resize((size_t)n);
    size_t bytes = align256(sys_table_bytes(n));
    for (int i = 0; i < n; ++i) {
        bf_status st = plan_image(descs[i], opts, &(*plans)[i]);
        if (st != BF_OK) return st;
        if ((*plans)[i].nch > 1) bytes += align256((size_t)descs[i].H * descs[i].W * sizeof(float));
    }
    *total = bytes;
    return BF_OK;
}

static bf_status prepare_v0(const bf_desc* descs, int n, const bf_opts* opts, void* workspace,
                            size_t ws_bytes, cudaStream_t stream) {
    const size_t need = v0_table_bytes(n);
    if (ws_bytes < need) return BF_ERR_NOMEM;
    std::vector<BatchImage> imgs((size_t)n);
    std::vector<long long> cost((size_t)n);
    for (int i = 0; i < n; ++i) {
        const bf_desc& d = descs[i];
        bf_opts o;
        if (opts) o = *opts; else bf_default_opts(&o);
        o.tile_w = 0;
        o.save_for_backward = 0;
        o.tile_h = v0_batch_rows(d.r < 0 ? 0 : d.r, opts);
        int nt = 0, gx = 0, gy = 0;
        bf_status st = fill_fwd_params(d.img, d.out, nullptr, d.H, d.W, d.pitch, d.r, d.sigma_r,
                                       d.T, d.N, &o, &imgs[i].p, &nt, &gx, &gy);
        if (st != BF_OK) return st;
        imgs[i].p.den = d.den;
        if (d.den && (d.den == d.out || (const void*)d.den == d.img)) return BF_ERR_INVALID_ARG;
        imgs[i].gx = gx;
        imgs[i].n_tiles = gx * gy;
        imgs[i].pad = 0;
        cost[i] = (long long)(imgs[i].p.Hb + 2 * d.r) * imgs[i].p.K;
    }
    std::vector<int> order((size_t)n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<char> host(need, 0);
    BatchTable* tab = reinterpret_cast<BatchTable*>(host.data());
    long long tiles = 0;
    for (int k = 0; k < n; ++k) {
        BatchImage bi = imgs[order[k]];
        bi.first_tile = (int)tiles;
        tiles += bi.n_tiles;
        if (tiles > (1LL << 30)) return BF_ERR_UNSUPPORTED;
        tab->img[k] = bi;
    }
    tab->n_tiles = (int)tiles;
    tab->n_images = n;
    tab->grid = sm_count();
    tab->kahan = opts ? opts->kahan : 0;
    tab->in_dtype = opts ? opts->in_dtype : BF_F32;
    cudaError_t e = cudaMemcpyAsync(workspace, host.data(), need, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return set_cuda_error(e);
    return BF_OK;
}

}  // namespace bf

using namespace bf;

extern "C" {

size_t bf_batch_workspace_bytes(const bf_desc* descs, int n, const bf_opts* opts) {
    if (!descs || n < 1 || check_opts(opts) != BF_OK) return 0;
    if (opts && opts->kahan) return v0_table_bytes(n);
    std::vector<Plan> plans;
    size_t total = 0;
    if (sys_layout(descs, n, opts, &plans, &total) != BF_OK) return 0;
    return total;
}

bf_status bf_batch_prepare(const bf_desc* descs, int n, const bf_opts* opts, void* workspace,
                           size_t ws_bytes, void* stream) {
    BF_TRACE("bf_batch_prepare");
    if (!descs || n < 1 || !workspace) return BF_ERR_INVALID_ARG;
    bf_status st = check_opts(opts);
    if (st != BF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (opts && opts->kahan) return prepare_v0(descs, n, opts, workspace, ws_bytes, s);

    std::vector<Plan> plans;
    size_t total = 0;
    st = sys_layout(descs, n, opts, &plans, &total);
    if (st != BF_OK) return st;
    if (ws_bytes < total) return BF_ERR_NOMEM;

    // groups in order (SysBatchTable::g); within a group the most expensive
    // tiles first
    std::vector<int> order((size_t)n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        if (plans[a].group != plans[b].group) return plans[a].group < plans[b].group;
        return plans[a].cost > plans[b].cost;
    });
    const size_t tbytes = sys_table_bytes(n);
    std::vector<char> host(tbytes, 0);
    SysBatchTable* tab = reinterpret_cast<SysBatchTable*>(host.data());
    tab->magic = SYS_BATCH_MAGIC;
    tab->in_dtype = opts ? opts->in_dtype : BF_F32;
    char* acc_base = static_cast<char*>(workspace) + align256(tbytes);
    size_t acc_off = 0;
    long long tiles[SYS_BATCH_GROUPS] = {};
    int count[SYS_BATCH_GROUPS] = {};
    for (int k = 0; k < n; ++k) {
        const int i = order[k];
        const Plan& pl = plans[i];
        const int grp = pl.group;
        SysBatchImage& im = tab->img[k];
        im.kind = pl.kind;
        im.nch = pl.nch;
        im.gx = pl.gx;
        im.n_tiles = pl.gx * pl.gy;
        im.first_tile = (int)tiles[grp];
        tiles[grp] += im.n_tiles;
        if (tiles[grp] > (1LL << 30)) return BF_ERR_UNSUPPORTED;
        if (count[grp]++ == 0) tab->g[grp].img0 = k;
        float* acc_den = nullptr;
        if (pl.nch > 1) {
            acc_den = reinterpret_cast<float*>(acc_base + acc_off);
            acc_off += align256((size_t)descs[i].H * descs[i].W * sizeof(float));
        }
        int per = (pl.p.K + pl.nch - 1) / pl.nch;
        per += per & 1;
        for (int c = 0; c < pl.nch; ++c) {
            const int i0 = c * per;
            const int kc = (pl.p.K - i0 < per) ? pl.p.K - i0 : per;
            SysParams& q = im.ch[c];
            memset(&q, 0, sizeof(q));
            q.img = pl.p.img;
            q.out = pl.p.out;
            q.dout = pl.p.den;
            q.acc_den = acc_den;
            q.H = pl.p.H; q.W = pl.p.W; q.r = pl.p.r;
            q.ld = pl.p.ld;
            q.K = kc;
            q.kstart = pl.p.kstart;
            q.Hb = pl.Hb;
            q.Tw = pl.wi - 2 * pl.p.r;
            q.k0 = pl.p.kstart + 2 * i0;
            q.acc = (pl.nch == 1) ? 0 : (c == 0 ? 1 : 3);
            q.gamma = pl.p.gamma;
            q.mid = pl.p.mid;
            q.gpi = (float)((double)pl.p.gamma / M_PI);
            for (int h = 0; h < kc; ++h) {
                q.a[h] = pl.p.a[i0 + h];
                q.ak[h] = pl.p.a[i0 + h] * (float)(pl.p.kstart + 2 * (i0 + h));
            }
            int kp = 1;
            while (2 * kp < kc) ++kp;
            im.kp[c] = kp <= 4 ? kp : (kp <= 6 ? 6 : (kp <= 8 ? 8 : SYS_KP_MAX));
        }
    }
    for (int grp = 0; grp < SYS_BATCH_GROUPS; ++grp) {
        tab->g[grp].n_tiles = (int)tiles[grp];
        tab->g[grp].n_images = count[grp];
        tab->g[grp].wi = grp == 2 ? 256 : 128;
    }
    cudaError_t e = cudaMemcpyAsync(workspace, host.data(), tbytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return set_cuda_error(e);
    return BF_OK;
}

bf_status bf_batch_launch(void* workspace, size_t ws_bytes, const bf_opts* opts, void* stream) {
    BF_TRACE("bf_batch_launch");
    if (!workspace) return BF_ERR_INVALID_ARG;
    bf_status st = check_opts(opts);
    if (st != BF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (opts && opts->kahan) {
        if (ws_bytes < sizeof(BatchTable)) return BF_ERR_INVALID_ARG;
        BatchTable* tab = static_cast<BatchTable*>(workspace);
        e = cudaMemsetAsync(&tab->counter, 0, sizeof(int), s);
        if (e == cudaSuccess) e = launch_batch(tab, sm_count(), 1, opts->in_dtype, s);
        if (e != cudaSuccess) return set_cuda_error(e);
        return BF_OK;
    }
    if (ws_bytes < sizeof(SysBatchTable)) return BF_ERR_INVALID_ARG;
    SysBatchTable* tab = static_cast<SysBatchTable*>(workspace);
    const int dtype = opts ? opts->in_dtype : BF_F32;
    e = cudaMemsetAsync(tab->counters, 0, sizeof(tab->counters), s);
    // one persistent launch per group, each with its resident CTAs; a group
    // with no tiles exits at its first pop
    for (int grp = 0; grp < SYS_BATCH_GROUPS && e == cudaSuccess; ++grp)
        e = launch_sys_batch(tab, grp, sys_batch_grid(grp, dtype), dtype, s);
    if (e != cudaSuccess) return set_cuda_error(e);
    return BF_OK;
}

bf_status bf_batch(const bf_desc* descs, int n, const bf_opts* opts, void* workspace,
                   size_t ws_bytes, void* stream) {
    bf_status st = bf_batch_prepare(descs, n, opts, workspace, ws_bytes, stream);
    if (st != BF_OK) return st;
    return bf_batch_launch(workspace, ws_bytes, opts, stream);
}

}  // extern "C"
