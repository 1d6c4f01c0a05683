// The C-ABI of libvrs: plan, the launch sequence of each step, and status.
#include <string.h>

#include "vrs_internal.cuh"

namespace vrs {
cudaError_t launch_preprocess(const ViewTable &vt, const DevScene &S, int scene, const int8_t *views,
                              int n_views, uint4 *pairs, float4 *rec, unsigned long long *keys,
                              uint32_t *vals, uint32_t *tile_cnt, DevStatus *st, unsigned long long cap,
                              float4 *viewtab, int64_t zero_tiles, float4 *raydepth, int n_sms,
                              cudaStream_t stream);
cudaError_t launch_sort(unsigned long long *keys0, uint32_t *vals0, unsigned long long *keys1,
                        uint32_t *vals1, uint32_t *counts, uint32_t *totals, uint2 *ranges,
                        int64_t n_tiles, const DevStatus *st, unsigned long long cap, int passes, int G,
                        int n_sms, cudaStream_t stream);
cudaError_t launch_tile_sort(const unsigned long long *keys_in, const uint32_t *vals_in,
                             unsigned long long *bucket, unsigned long long *keys_out, uint32_t *vals_out,
                             const uint32_t *cnt, uint32_t *cursor, uint32_t *blocksum, uint32_t *big_list,
                             uint2 *ranges, DevStatus *st, unsigned long long cap, int64_t n_tiles,
                             uint32_t blend_max, int n_sms, cudaStream_t s);
cudaError_t launch_render_fwd(const ViewTable &vt, const float4 *viewtab, const float4 *rec,
                              const uint32_t *vals, const uint2 *ranges, DevStatus *st, float *rgb,
                              float *depth, float *Tf, uint32_t *ncontrib, uint32_t *tile_work, uint32_t *order,
                              uint32_t *order_tmp, int64_t n_tiles, int64_t n_records,
                              unsigned long long cap, int persistent, int count, int half_out,
                              int tiles_per_pull, const unsigned long long *bucket,
                              unsigned long long *keys_w, uint32_t *vals_w, uint32_t blend_max, int n_sms,
                              cudaStream_t s);
cudaError_t launch_render_resort(const ViewTable &vt, const float4 *viewtab, const float4 *rec,
                                 const float4 *raydepth, const uint32_t *vals, const uint2 *ranges,
                                 DevStatus *st, float *rgb, float *depth, float *Tf, uint8_t *flags,
                                 int64_t n_tiles, int64_t n_records, unsigned long long cap, int window,
                                 int half_out, cudaStream_t s);
cudaError_t launch_render_bwd(const ViewTable &vt, const float4 *viewtab, const float4 *rec,
                              const uint32_t *vals, const uint2 *ranges, const DevStatus *st,
                              const uint32_t *ncontrib, const float *Tf, const float *dL_drgb,
                              const float *dL_ddepth, const float *dL_dT, float *grad2d, const uint32_t *order,
                              int64_t n_tiles, int64_t n_records, unsigned long long cap, cudaStream_t s);
cudaError_t launch_tile_order(const uint2 *ranges, const uint32_t *work, int wpt, int64_t n_tiles,
                              const DevStatus *st, uint32_t *order, uint32_t *order_tmp, int n_sms, bool clear_tmp,
                              cudaStream_t s);
cudaError_t launch_clear_pair_rows(const uint4 *pairs, const DevStatus *st, int scene, int64_t n_gauss,
                                   int64_t rec_base, float *grad2d, int n_sms, cudaStream_t s);
cudaError_t launch_backward_params(const ViewTable &vt, const DevScene &S, const DevScene &G,
                                   const int8_t *views, int n_views, const float *grad2d, DevStatus *st,
                                   uint32_t *list, const uint4 *pairs, int scene, int n_sms, cudaStream_t s);
}  // namespace vrs

using namespace vrs;

namespace {

constexpr int kOrderTmp = 2 * kOrderBuckets;   // histogram + cursors of the work-order buckets

// Warps of a blend CTA: entries per tile of the reverse pass's work estimate.
int warps_per_tile(int tile) { return tile * tile / 64; }

// Backward plans: the reverse pass's per-warp work estimates, written by the
// forward, take the workspace's last region (its offset follows from the size).
int64_t work_bytes(const vrs_plan &P) { return P.n_tiles * warps_per_tile(P.tile) * 4; }

int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

int bits_for(int64_t n)
{
    int b = 1;
    while (b < 40 && ((int64_t)1 << b) < n) ++b;
    return b;
}

vrs_status cuda_status(cudaError_t e) { return e == cudaSuccess ? VRS_OK : VRS_ERR_CUDA; }

uint32_t *work_estimates(const vrs_plan *P, void *workspace)
{
    return reinterpret_cast<uint32_t *>(static_cast<char *>(workspace) + P->workspace_bytes -
                                        align_up(work_bytes(*P), 256));
}

template <typename T>
T *at(void *ws, int64_t off) { return reinterpret_cast<T *>(static_cast<char *>(ws) + off); }

void fill_sizes(const vrs_plan *P, ViewTable &vt)
{
    memset(&vt, 0, sizeof(vt));
    vt.n_views = P->n_views;
    vt.tile = P->tile;
    for (int v = 0; v < P->n_views; ++v) {
        DevView &d = vt.v[v];
        d.w = P->view_w[v];
        d.h = P->view_h[v];
        d.gw = P->view_gw[v];
        d.gh = P->view_gh[v];
        d.scene = P->view_scene[v];
        d.rec_base = P->view_rec_base[v];
        d.tile_base = P->view_tile_base[v];
        d.pix_base = P->view_pix_base[v];
    }
}

vrs_status fill_cameras(const vrs_plan *P, const vrs_camera *views, ViewTable &vt)
{
    if (!views) return VRS_ERR_INVALID;
    for (int v = 0; v < P->n_views; ++v) {
        const vrs_camera &c = views[v];
        if (c.width != P->view_w[v] || c.height != P->view_h[v] || c.scene != P->view_scene[v])
            return VRS_ERR_INVALID;
        if (!(c.fx > 0.f) || !(c.fy > 0.f) || !(c.znear >= 0.f)) return VRS_ERR_INVALID;
        DevView &d = vt.v[v];
        memcpy(d.R, c.R, sizeof(d.R));
        memcpy(d.t, c.t, sizeof(d.t));
        d.fx = c.fx;
        d.fy = c.fy;
        d.cx = c.cx;
        d.cy = c.cy;
        d.znear = c.znear;
        d.tanx = c.tan_fovx > 0.f ? c.tan_fovx : (float)c.width / (2.0f * c.fx);
        d.tany = c.tan_fovy > 0.f ? c.tan_fovy : (float)c.height / (2.0f * c.fy);
    }
    return VRS_OK;
}

vrs_status check_scenes(const vrs_plan *P, const vrs_scene *scenes)
{
    if (!scenes) return VRS_ERR_INVALID;
    for (int s = 0; s < P->n_scenes; ++s) {
        const vrs_scene &S = scenes[s];
        if (S.n != P->scene_n[s] || S.sh_degree != P->scene_deg[s]) return VRS_ERR_INVALID;
        if (S.n > 0 && (!S.means || !S.sh)) return VRS_ERR_INVALID;
        if (S.n > 0 && !S.baked && (!S.log_scales || !S.quats || !S.opacity_logits)) return VRS_ERR_INVALID;
        if (S.baked && (reinterpret_cast<uintptr_t>(S.baked) & 15u)) return VRS_ERR_INVALID;
    }
    return VRS_OK;
}

DevScene dev_scene(const vrs_scene &S)
{
    DevScene d;
    d.means = S.means;
    d.log_scales = S.log_scales;
    d.quats = S.quats;
    d.logits = S.opacity_logits;
    d.sh = S.sh;
    d.baked = reinterpret_cast<const float4 *>(S.baked);
    d.n = S.n;
    d.K = (S.sh_degree + 1) * (S.sh_degree + 1);
    d.sh_half = S.sh_half ? 1 : 0;
    return d;
}

// Sort mode 2: tiles of at most one blend batch (tile^2 / 2 instances) are ordered by the blend.
uint32_t blend_sorted_max(const vrs_plan *P)
{
    return P->sort_mode == 2 ? (uint32_t)(P->tile * P->tile / 2) : 0u;
}

int views_of_scene(const vrs_plan *P, int s, int8_t *out)
{
    int n = 0;
    for (int v = 0; v < P->n_views; ++v)
        if (P->view_scene[v] == s) out[n++] = (int8_t)v;
    return n;
}

// Backward plans whose reverse pass reads only the visible pairs' 2D-gradient rows: every
// scene with Gaussians has one view, and the touched-Gaussian list fits the spare
// record-index buffer (so the pair list survives for it).
bool pair_grads(const vrs_plan *P)
{
    if (!P->backward || P->max_instances < P->n_records) return false;
    for (int s = 0; s < P->n_scenes; ++s) {
        int8_t vl[VRS_MAX_VIEWS];
        if (P->scene_n[s] > 0 && views_of_scene(P, s, vl) > 1) return false;
    }
    return true;
}

}  // namespace

extern "C" {

vrs_status vrs_plan_batch(const vrs_scene *scenes, int32_t n_scenes, const vrs_camera *views,
                          int32_t n_views, const vrs_plan_opts *opts, vrs_plan *plan)
{
    if (!plan || !scenes || !views) return VRS_ERR_INVALID;
    if (n_views < 1 || n_views > VRS_MAX_VIEWS || n_scenes < 1 || n_scenes > VRS_MAX_SCENES)
        return VRS_ERR_INVALID;
    vrs_plan_opts o;
    memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    const int tile = o.tile == 0 ? 16 : o.tile;
    if (tile != 8 && tile != 16 && tile != 32) return VRS_ERR_INVALID;
    if (o.max_instances < 0) return VRS_ERR_INVALID;
    if (o.sort != 0 && o.sort != 1 && o.sort != 2) return VRS_ERR_INVALID;
    if (o.sort == 2 && o.resort) return VRS_ERR_INVALID;     // the window kernel reads sorted lists
    if (o.resort != 0 && o.resort != 4 && o.resort != 8 && o.resort != 16) return VRS_ERR_INVALID;
    if (o.resort && (o.backward || (tile == 32 && o.resort > 8))) return VRS_ERR_INVALID;
    if (o.half_out && o.backward) return VRS_ERR_INVALID;
    if (o.tiles_per_pull < 0 || o.tiles_per_pull > 64) return VRS_ERR_INVALID;
    if (o.persistent < 0 || o.persistent > 2) return VRS_ERR_INVALID;
    if (o.key_bits < 0 || o.key_bits > 64) return VRS_ERR_INVALID;
    vrs_plan P;
    memset(&P, 0, sizeof(P));
    P.n_views = n_views;
    P.n_scenes = n_scenes;
    P.tile = tile;
    P.persistent = o.persistent;
    P.backward = o.backward ? 1 : 0;
    P.sort_mode = o.sort;
    P.count_pairs = o.count_pairs ? 1 : 0;
    P.resort = o.resort;
    P.half_out = o.half_out ? 1 : 0;
    P.tiles_per_pull = o.tiles_per_pull > 0 ? o.tiles_per_pull : 1;
    for (int s = 0; s < n_scenes; ++s) {
        if (scenes[s].n < 0 || scenes[s].sh_degree < 0 || scenes[s].sh_degree > 3) return VRS_ERR_INVALID;
        P.scene_n[s] = scenes[s].n;
        P.scene_deg[s] = scenes[s].sh_degree;
    }
    int64_t rec = 0, tiles = 0, pix = 0;
    for (int v = 0; v < n_views; ++v) {
        const vrs_camera &c = views[v];
        if (c.width < 1 || c.height < 1 || c.width > 16384 || c.height > 16384) return VRS_ERR_INVALID;
        if (c.scene < 0 || c.scene >= n_scenes) return VRS_ERR_INVALID;
        P.view_scene[v] = c.scene;
        P.view_w[v] = c.width;
        P.view_h[v] = c.height;
        P.view_gw[v] = (c.width + tile - 1) / tile;
        P.view_gh[v] = (c.height + tile - 1) / tile;
        P.view_rec_base[v] = rec;
        P.view_tile_base[v] = tiles;
        P.view_pix_base[v] = pix;
        rec += P.scene_n[c.scene];
        tiles += (int64_t)P.view_gw[v] * P.view_gh[v];
        pix += (int64_t)c.width * c.height;
    }
    if (rec >= ((int64_t)1 << 32) || tiles >= ((int64_t)1 << 31)) return VRS_ERR_INVALID;
    P.n_records = rec;
    P.n_tiles = tiles;
    P.n_pixels = pix;
    P.key_bits = 32 + bits_for(tiles);
    if (o.key_bits) {                     // a wider radix key: more passes, the same order
        if (o.key_bits < P.key_bits) return VRS_ERR_INVALID;
        P.key_bits = o.key_bits;
    }
    P.sort_passes = (P.key_bits + 7) / 8;
    P.sorted_buf = P.sort_mode == 1 ? P.sort_passes % 2 : 0;
    int64_t cap = o.max_instances > 0 ? o.max_instances : 4 * rec + 65536;
    if (cap > ((int64_t)1 << 31)) cap = (int64_t)1 << 31;
    P.max_instances = cap;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
        cudaGetLastError();
        sms = 152;
    }
    P.n_sms = sms;
    P.sort_ctas = 2 * sms > 1024 ? 1024 : 2 * sms;
    // workspace layout
    int64_t off = 0;
    auto take = [&](int64_t bytes) {
        int64_t r = off;
        off = align_up(off + (bytes > 0 ? bytes : 1), 256);
        return r;
    };
    P.off_status = take(256 + sizeof(float4) * VRS_MAX_VIEWS);   // status + device view table
    P.off_records = take(rec * kRecF4 * 16);
    P.off_keys[0] = take(cap * 8);
    P.off_keys[1] = take(cap * 8);
    P.off_vals[0] = take(cap * 4);
    P.off_vals[1] = take(cap * 4);
    P.off_hist = take(((int64_t)256 * P.sort_ctas + 256) * 4);
    P.off_ranges = take(tiles * 8);
    P.off_ncontrib = take(pix * 4);
    P.off_order = take((tiles + kOrderTmp) * 4);
    P.off_grad2d = P.backward ? take(rec * kGrad2D * 4) : 0;
    P.off_tilesort = take((3 * tiles + (tiles + 1023) / 1024) * 4);
    P.off_pairs = take(rec * 32);
    P.off_raydepth = P.resort ? take(rec * 3 * 16) : 0;
    P.off_resort_flags = P.resort ? take(pix) : 0;
    if (P.backward) take(work_bytes(P));   // the last region (see work_estimates)
    P.workspace_bytes = off;
    *plan = P;
    return VRS_OK;
}

vrs_status vrs_preprocess(const vrs_plan *plan, const vrs_scene *scenes, const vrs_camera *views,
                          void *workspace, void *stream)
{
    if (!plan || !workspace) return VRS_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(workspace) & 255u) return VRS_ERR_INVALID;
    vrs_status vs = check_scenes(plan, scenes);
    if (vs != VRS_OK) return vs;
    ViewTable vt;
    fill_sizes(plan, vt);
    vs = fill_cameras(plan, views, vt);
    if (vs != VRS_OK) return vs;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevStatus *st = at<DevStatus>(workspace, plan->off_status);
    float4 *viewtab = at<float4>(workspace, plan->off_status + 256);
    cudaError_t e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
    if (e != cudaSuccess) return VRS_ERR_CUDA;
    // the per-tile counts of the bucketed sort are cleared by the first scene's
    // decision kernel (before any pair kernel counts into them), or here when no
    // scene has Gaussians
    uint32_t *tile_cnt = nullptr;
    int first = -1;
    if (plan->sort_mode != 1) {
        tile_cnt = at<uint32_t>(workspace, plan->off_tilesort);
        for (int sc = 0; sc < plan->n_scenes && first < 0; ++sc)
            if (plan->scene_n[sc] > 0) {
                int8_t vl[VRS_MAX_VIEWS];
                if (views_of_scene(plan, sc, vl) > 0) first = sc;
            }
        if (first < 0) {
            e = cudaMemsetAsync(tile_cnt, 0, sizeof(uint32_t) * (size_t)plan->n_tiles, s);
            if (e != cudaSuccess) return VRS_ERR_CUDA;
        }
    }
    int64_t pair_base = 0;
    for (int sc = 0; sc < plan->n_scenes; ++sc) {
        int8_t vlist[VRS_MAX_VIEWS];
        const int nv = views_of_scene(plan, sc, vlist);
        e = launch_preprocess(vt, dev_scene(scenes[sc]), sc, vlist, nv,
                              at<uint4>(workspace, plan->off_pairs) + 2 * pair_base,
                              at<float4>(workspace, plan->off_records),
                              at<unsigned long long>(workspace, plan->off_keys[0]),
                              at<uint32_t>(workspace, plan->off_vals[0]), tile_cnt, st,
                              (unsigned long long)plan->max_instances, viewtab,
                              sc == first ? plan->n_tiles : 0,
                              plan->resort ? at<float4>(workspace, plan->off_raydepth) : nullptr, plan->n_sms, s);
        if (e != cudaSuccess) return VRS_ERR_CUDA;
        pair_base += (int64_t)plan->scene_n[sc] * nv;
    }
    return VRS_OK;
}

vrs_status vrs_bin_sort(const vrs_plan *plan, void *workspace, void *stream)
{
    if (!plan || !workspace) return VRS_ERR_INVALID;
    if (plan->sort_mode != 1) {
        uint32_t *ts = at<uint32_t>(workspace, plan->off_tilesort);
        const int64_t nt = plan->n_tiles;
        cudaError_t e = launch_tile_sort(
            at<unsigned long long>(workspace, plan->off_keys[0]), at<uint32_t>(workspace, plan->off_vals[0]),
            at<unsigned long long>(workspace, plan->off_keys[1]), at<unsigned long long>(workspace, plan->off_keys[0]),
            at<uint32_t>(workspace, plan->off_vals[0]), ts, ts + nt, ts + 3 * nt, ts + 2 * nt,
            at<uint2>(workspace, plan->off_ranges), at<DevStatus>(workspace, plan->off_status),
            (unsigned long long)plan->max_instances, nt, blend_sorted_max(plan), plan->n_sms,
            static_cast<cudaStream_t>(stream));
        return cuda_status(e);
    }
    uint32_t *hist = at<uint32_t>(workspace, plan->off_hist);
    cudaError_t e = launch_sort(at<unsigned long long>(workspace, plan->off_keys[0]),
                                at<uint32_t>(workspace, plan->off_vals[0]),
                                at<unsigned long long>(workspace, plan->off_keys[1]),
                                at<uint32_t>(workspace, plan->off_vals[1]), hist,
                                hist + (size_t)256 * plan->sort_ctas,
                                at<uint2>(workspace, plan->off_ranges), plan->n_tiles,
                                at<DevStatus>(workspace, plan->off_status),
                                (unsigned long long)plan->max_instances, plan->sort_passes,
                                plan->sort_ctas, plan->n_sms, static_cast<cudaStream_t>(stream));
    return cuda_status(e);
}

vrs_status vrs_render_fwd(const vrs_plan *plan, void *workspace, float *rgb, float *depth,
                          float *T_final, void *stream)
{
    if (!plan || !workspace || !rgb || !depth || !T_final) return VRS_ERR_INVALID;
    ViewTable vt;
    fill_sizes(plan, vt);
    const int sb = plan->sorted_buf;
    if (plan->resort) {
        return cuda_status(launch_render_resort(
            vt, at<float4>(workspace, plan->off_status + 256), at<float4>(workspace, plan->off_records),
            at<float4>(workspace, plan->off_raydepth), at<uint32_t>(workspace, plan->off_vals[sb]),
            at<uint2>(workspace, plan->off_ranges), at<DevStatus>(workspace, plan->off_status), rgb, depth,
            T_final, at<uint8_t>(workspace, plan->off_resort_flags), plan->n_tiles, plan->n_records,
            (unsigned long long)plan->max_instances, plan->resort, plan->half_out,
            static_cast<cudaStream_t>(stream)));
    }
    uint32_t *order = at<uint32_t>(workspace, plan->off_order);
    cudaError_t e = launch_render_fwd(
        vt, at<float4>(workspace, plan->off_status + 256), at<float4>(workspace, plan->off_records),
        at<uint32_t>(workspace, plan->off_vals[sb]), at<uint2>(workspace, plan->off_ranges),
        at<DevStatus>(workspace, plan->off_status), rgb, depth, T_final,
        plan->backward ? at<uint32_t>(workspace, plan->off_ncontrib) : nullptr,   // only the reverse pass reads it
        plan->backward ? work_estimates(plan, workspace) : nullptr, order, order + plan->n_tiles, plan->n_tiles,
        plan->n_records, (unsigned long long)plan->max_instances, plan->persistent,
        plan->half_out ? 0 : plan->count_pairs, plan->half_out, plan->tiles_per_pull,
        at<unsigned long long>(workspace, plan->off_keys[1]), at<unsigned long long>(workspace, plan->off_keys[sb]),
        at<uint32_t>(workspace, plan->off_vals[sb]), blend_sorted_max(plan), plan->n_sms,
        static_cast<cudaStream_t>(stream));
    return cuda_status(e);
}

vrs_status vrs_render_bwd(const vrs_plan *plan, void *workspace, const vrs_scene *scenes,
                          const vrs_camera *views, const float *T_final, const float *dL_drgb,
                          const float *dL_ddepth, const float *dL_dT, const vrs_scene *grads,
                          void *stream)
{
    if (!plan || !workspace || !T_final || !dL_drgb || !dL_ddepth || !grads) return VRS_ERR_INVALID;
    if (!plan->backward) return VRS_ERR_INVALID;
    vrs_status vs = check_scenes(plan, scenes);
    if (vs != VRS_OK) return vs;
    for (int s = 0; s < plan->n_scenes; ++s)      // the reverse pass needs the parameter form in FP32
        if (scenes[s].baked || scenes[s].sh_half) return VRS_ERR_INVALID;
    for (int s = 0; s < plan->n_scenes; ++s) {
        const vrs_scene &G = grads[s];
        if (G.n != plan->scene_n[s] || G.sh_degree != plan->scene_deg[s]) return VRS_ERR_INVALID;
        if (G.n > 0 && (!G.means || !G.log_scales || !G.quats || !G.opacity_logits || !G.sh))
            return VRS_ERR_INVALID;
    }
    ViewTable vt;
    fill_sizes(plan, vt);
    vs = fill_cameras(plan, views, vt);
    if (vs != VRS_OK) return vs;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float *g2 = at<float>(workspace, plan->off_grad2d);
    const DevStatus *st = at<DevStatus>(workspace, plan->off_status);
    // the work order's scratch first, so that the clearing, order and reverse-pass kernels
    // follow one another without a memset between them
    uint32_t *order = at<uint32_t>(workspace, plan->off_order);
    cudaError_t e = cudaMemsetAsync(order + plan->n_tiles, 0, sizeof(uint32_t) * kOrderTmp, s);
    if (e != cudaSuccess) return VRS_ERR_CUDA;
    if (pair_grads(plan)) {
        // every scene has one view: only its visible pairs' rows are read, and cleared
        int64_t pb = 0;
        for (int sc = 0; sc < plan->n_scenes; ++sc) {
            int8_t vl[VRS_MAX_VIEWS];
            const int nv = views_of_scene(plan, sc, vl);
            if (nv == 1) {
                e = launch_clear_pair_rows(at<uint4>(workspace, plan->off_pairs) + 2 * pb, st, sc, plan->scene_n[sc],
                                           plan->view_rec_base[vl[0]], g2, plan->n_sms, s);
                if (e != cudaSuccess) return VRS_ERR_CUDA;
            }
            pb += (int64_t)plan->scene_n[sc] * nv;
        }
    } else {
        e = cudaMemsetAsync(g2, 0, sizeof(float) * kGrad2D * (size_t)plan->n_records, s);
        if (e != cudaSuccess) return VRS_ERR_CUDA;
    }
    // heaviest tiles first, so that the last wave holds no long tile
    e = launch_tile_order(at<uint2>(workspace, plan->off_ranges), work_estimates(plan, workspace),
                          warps_per_tile(plan->tile), plan->n_tiles, st, order, order + plan->n_tiles, plan->n_sms,
                          false, s);
    if (e != cudaSuccess) return VRS_ERR_CUDA;
    e = launch_render_bwd(vt, at<float4>(workspace, plan->off_status + 256),
                          at<float4>(workspace, plan->off_records),
                          at<uint32_t>(workspace, plan->off_vals[plan->sorted_buf]),
                          at<uint2>(workspace, plan->off_ranges), st,
                          at<uint32_t>(workspace, plan->off_ncontrib), T_final, dL_drgb, dL_ddepth,
                          dL_dT, g2, order, plan->n_tiles, plan->n_records, (unsigned long long)plan->max_instances, s);
    if (e != cudaSuccess) return VRS_ERR_CUDA;
    // the touched-Gaussian list goes to the record-index buffer the sort left unused (when
    // it holds a record index per record), so that the forward's pair list stays intact and
    // one-view scenes can list their touched Gaussians from it; else to the pair-list area
    const bool list_in_vals = plan->max_instances >= plan->n_records;
    uint32_t *list = list_in_vals ? at<uint32_t>(workspace, plan->off_vals[1 - plan->sorted_buf])
                                  : at<uint32_t>(workspace, plan->off_pairs);
    int64_t pair_base = 0;
    for (int sc = 0; sc < plan->n_scenes; ++sc) {
        int8_t vlist[VRS_MAX_VIEWS];
        const int nv = views_of_scene(plan, sc, vlist);
        e = launch_backward_params(vt, dev_scene(scenes[sc]), dev_scene(grads[sc]), vlist, nv, g2,
                                   at<DevStatus>(workspace, plan->off_status), list,
                                   list_in_vals ? at<uint4>(workspace, plan->off_pairs) + 2 * pair_base : nullptr,
                                   sc, plan->n_sms, s);
        if (e != cudaSuccess) return VRS_ERR_CUDA;
        pair_base += (int64_t)plan->scene_n[sc] * nv;
    }
    return VRS_OK;
}

vrs_status vrs_query_status(const vrs_plan *plan, const void *workspace, vrs_run_info *info,
                            void *stream)
{
    if (!plan || !workspace) return VRS_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    vrs_run_info h;
    memset(&h, 0, sizeof(h));
    cudaError_t e = cudaMemcpyAsync(&h, static_cast<const char *>(workspace) + plan->off_status,
                                    sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return VRS_ERR_CUDA;
    if (info) *info = h;
    if (h.flags & ST_CAPACITY) return VRS_ERR_CAPACITY;
    if (h.flags & ST_TIMEOUT) return VRS_ERR_TIMEOUT;
    if (h.flags & ST_NONFINITE) return VRS_ERR_NONFINITE;
    if (h.flags & ST_ZERO_QUAT) return VRS_ERR_INVALID;
    return VRS_OK;
}

vrs_status vrs_reset_status(const vrs_plan *plan, void *workspace, void *stream)
{
    if (!plan || !workspace) return VRS_ERR_INVALID;
    return cuda_status(cudaMemsetAsync(static_cast<char *>(workspace) + plan->off_status, 0,
                                       sizeof(DevStatus), static_cast<cudaStream_t>(stream)));
}

const char *vrs_status_string(vrs_status status)
{
    switch (status) {
        case VRS_OK: return "VRS_OK";
        case VRS_ERR_INVALID: return "VRS_ERR_INVALID";
        case VRS_ERR_CAPACITY: return "VRS_ERR_CAPACITY";
        case VRS_ERR_CUDA: return "VRS_ERR_CUDA";
        case VRS_ERR_TIMEOUT: return "VRS_ERR_TIMEOUT";
        case VRS_ERR_NONFINITE: return "VRS_ERR_NONFINITE";
    }
    return "VRS_ERR_UNKNOWN";
}

}  // extern "C"
