// Host side of the batched entry points: builds the tile table of many
// uneven images (each with its own r, N, gamma, a_k) in the caller's
// workspace and launches the persistent tile-queue kernel.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "bf_internal.cuh"

namespace bf {

// Rows per band in a batch: small enough that the queue balances the
// load of 256 uneven images over the SMs, tall enough that the 2r warm-up
// rows of each band stay a minor cost.
static int batch_band_rows(int r, const bf_opts* o) {
    if (o && o->tile_h > 0) return o->tile_h;
    int hb = 128;
    if (hb < 4 * r) hb = 4 * r;
    return hb;
}

static size_t table_bytes(int n) {
    return sizeof(BatchTable) + (size_t)(n > 1 ? n - 1 : 0) * sizeof(BatchImage);
}

}  // namespace bf

using namespace bf;

extern "C" {

size_t bf_batch_workspace_bytes(const bf_desc* descs, int n, const bf_opts* opts) {
    (void)descs;
    (void)opts;
    if (n < 1) return 0;
    return table_bytes(n);
}

bf_status bf_batch_prepare(const bf_desc* descs, int n, const bf_opts* opts, void* workspace,
                           size_t ws_bytes, void* stream) {
    if (!descs || n < 1 || !workspace) return BF_ERR_INVALID_ARG;
    bf_status st = check_opts(opts);
    if (st != BF_OK) return st;
    const size_t need = table_bytes(n);
    if (ws_bytes < need) return BF_ERR_NOMEM;
    std::vector<BatchImage> imgs((size_t)n);
    std::vector<long long> cost((size_t)n);
    for (int i = 0; i < n; ++i) {
        const bf_desc& d = descs[i];
        bf_opts o;
        if (opts) o = *opts; else bf_default_opts(&o);
        o.tile_w = 0;  // the batch kernel always runs 256-thread strips
        o.save_for_backward = 0;
        o.tile_h = batch_band_rows(d.r < 0 ? 0 : d.r, opts);
        int nt = 0, gx = 0, gy = 0;
        st = fill_fwd_params(d.img, d.out, nullptr, d.H, d.W, d.r, d.sigma_r, d.T, d.N, &o,
                             &imgs[i].p, &nt, &gx, &gy);
        if (st != BF_OK) return st;
        imgs[i].gx = gx;
        imgs[i].n_tiles = gx * gy;
        imgs[i].pad = 0;
        // per-tile cost ~ (band rows + warm-up) x harmonics
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
    tab->counter = 0;
    tab->n_tiles = (int)tiles;
    tab->n_images = n;
    tab->grid = sm_count();
    tab->kahan = opts ? opts->kahan : 0;
    tab->in_dtype = opts ? opts->in_dtype : BF_F32;
    cudaError_t e = cudaMemcpyAsync(workspace, host.data(), need, cudaMemcpyHostToDevice,
                                    (cudaStream_t)stream);
    if (e != cudaSuccess) return set_cuda_error(e);
    return BF_OK;
}

bf_status bf_batch_launch(void* workspace, size_t ws_bytes, const bf_opts* opts, void* stream) {
    if (!workspace || ws_bytes < sizeof(BatchTable)) return BF_ERR_INVALID_ARG;
    bf_status st = check_opts(opts);
    if (st != BF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    BatchTable* tab = static_cast<BatchTable*>(workspace);
    cudaError_t e = cudaMemsetAsync(&tab->counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return set_cuda_error(e);
    e = launch_batch(tab, sm_count(), opts ? opts->kahan : 0, opts ? opts->in_dtype : BF_F32, s);
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
