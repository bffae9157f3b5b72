// psfs_api.cu -- host side of libpsfs: the C ABI declared in include/psfs.h.
//
// Argument checking, handle state, device scratch, and the order of the
// kernel launches of each call.  No arithmetic of the method runs here
// beyond the per-camera projection matrices and scalar constants, which are
// formed once in double precision at handle creation.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "psfs_internal.cuh"

using namespace psfs;

// Device staging slots of the host-buffer sequence path.
constexpr int kIoSlots = 3;
// Candidates of psfs_batch_autotune.
constexpr int kBatchCandidates = PSFS_N_BATCH_CANDIDATES;
// Streams of the batch's graph of per-frame launches.
constexpr int kBatchStreams = 4;


struct psfs_handle {
    int device = 0;
    cudaStream_t stream = nullptr;
    psfs_grid grid{};
    std::vector<psfs_camera> cams;
    int n_cams = 0;
    int W = 0, H = 0;
    psfs_params params{};
    int64_t n_pix = 0;          // n_cams * H * W
    size_t map_elem = 4;

    SensorConsts sc{};
    float c0 = 0.0f;
    FuseArgs fuse{};            // per-call pointers filled in at launch
    FuseShape shape = kDefaultFuseShape;

    void *maps = nullptr;       // [n_cams][H][W] of g
    CUtensorMap tm_main[kBoxClasses];   // tensor maps of `maps` (staged kernel)
    CUtensorMap tm_alt[kBoxClasses];    // tensor maps of `maps2` (sequence path)
    bool tm_main_ok = false, tm_alt_ok = false;
    float *bg_mean = nullptr;   // [n_pix][3]  } one allocation, so that one L2
    float *bg_hinv = nullptr;   // [n_pix][3]  } access window covers both
    bool bg_l2 = false;         // keep the background resident in L2 (sequence path)
    bool bg_ready = false;
    uint32_t *d_words = nullptr;    // [0] status, [1] scratch counter, [2] host-path count
    uint32_t *h_words = nullptr;    // pinned mirror
    uint64_t *tiles = nullptr;
    int4 *tilecam = nullptr;    // [n_tiles][n_cams] staging records
    int n_tiles = 0;

    // host-buffer path staging (allocated on first use)
    uint8_t *st_images = nullptr;
    float *st_occ = nullptr;
    uint32_t *st_list = nullptr;
    uint32_t st_list_cap = 0;

    // sequence path: likelihood and fusion of consecutive frames on two
    // streams, maps double-buffered (created on first use)
    cudaStream_t seq_stream[2] = {nullptr, nullptr};   // [0] likelihood, [1] fusion
    cudaEvent_t seq_ev_in = nullptr, seq_ev_map[2] = {nullptr, nullptr}, seq_ev_fused[2] = {nullptr, nullptr};
    cudaEvent_t seq_ev_done[2] = {nullptr, nullptr};
    void *maps2 = nullptr;
    int seq_lk_ctas = 2;
    // frame groups: frames per group on the sequence path (1 = one frame per
    // launch) and the two group map buffers [n_pix][group_cap] (first use)
    int seq_group = 1;
    int seq_rec = 32;   // bytes per pixel record of a group's map planes (32 or 64)
    void *gmaps[2] = {nullptr, nullptr};
    int group_cap = 0;
    // the sequence path's own tile shape and plan (seq_own), when it differs
    // from `shape` (the autotuner keeps the best shape for one frame per call
    // in `shape` and the best one for frame groups here)
    bool seq_own = false;
    FuseShape seq_shape = kDefaultFuseShape;
    uint64_t *seq_tiles = nullptr;
    int4 *seq_tilecam = nullptr;
    int seq_n_tiles = 0;

    // host-buffer sequence path (first use): kIoSlots chunk slots of device
    // staging, copies in and out on two streams of their own
    cudaStream_t io_stream[2] = {nullptr, nullptr};   // [0] host to device, [1] device to host
    cudaEvent_t io_ev_in[kIoSlots] = {}, io_ev_comp[kIoSlots] = {};
    cudaEvent_t io_ev_cnt[kIoSlots] = {}, io_ev_out[kIoSlots] = {};
    uint8_t *io_img[kIoSlots] = {};
    float *io_occ[kIoSlots] = {};
    uint32_t *io_list[kIoSlots] = {};
    uint32_t *io_cnt[kIoSlots] = {};
    int io_frames = 0;          // frames per slot
    uint32_t io_cap = 0;        // list entries per frame

    // inner-voxel removal: per-frame occupancy bitmasks (first use)
    uint32_t *surf_masks = nullptr;
    int surf_frames = 0;

    // tracing: CUDA event pairs around each launch
    int prof_cap = 0;
    std::vector<cudaEvent_t> prof_ev;      // 2 * prof_cap events
    std::vector<int> prof_stage;           // stage of each recorded pair
    int prof_n = 0;

    // adjoint scratch (allocated on first use)
    float *dl = nullptr;        // [n_vox] dLoss / dlogodds
    float *dl_rec = nullptr;    // [2][n_vox][kBwRecord] the same for psfs_backward_sequence
    float *dl_rec2 = nullptr;   // its second buffer: group g's records in buffer g & 1
    // owner lists of the pixel pass (built by the first adjoint call): pixel
    // p owns own_vox[own_off[p] .. own_off[p + 1])
    uint32_t *own_off = nullptr;   // [n_pix + 1]
    uint32_t *own_vox = nullptr;   // [n_vox * n_cams] (upper bound of the pairs)
    uint32_t *own_cnt = nullptr;   // [n_pix] counts, then fill cursors
    uint32_t *own_sums = nullptr;  // block totals of the offset scan
    bool own_ready = false;
    // batched adjoint (psfs_backward_sequence, first use): its own tile plan
    // in the shape of the frame-group kernels, and maps of up to kBwRecord
    // frames as one plane of records [n_pix][frames]
    FuseArgs bw_fuse{};
    uint64_t *bw_tiles = nullptr;
    int4 *bw_tilecam = nullptr;
    void *bw_maps = nullptr;
};

namespace psfs {

namespace {
thread_local std::string g_last_error;
}  // namespace

psfs_status record_failure(psfs_status s, const char *what)
{
    g_last_error = what;
    return s;
}

psfs_status record_cuda_failure(cudaError_t e, const char *where)
{
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return PSFS_ERR_CUDA;
}

const char *last_failure() { return g_last_error.c_str(); }

int device_sm_count()
{
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 1;   // grid-stride launches stay correct with any grid size
    }
    if (!cached[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) cudaGetLastError();
        cached[dev] = n > 0 ? n : 1;
    }
    return cached[dev];
}

}  // namespace psfs

namespace {

psfs_status fail(psfs_status s, const char *what) { return psfs::record_failure(s, what); }

psfs_status fail_cuda(cudaError_t e, const char *where) { return psfs::record_cuda_failure(e, where); }

#define PSFS_CK(call)                                                  \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return fail_cuda(e_, #call);            \
    } while (0)

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

bool finite_all(const double *v, int n)
{
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

// Floats of each half (mean, then 1 / (2 var)) of the background
// allocation: 3 per pixel rounded up to 256 bytes, so that the second half
// starts on a boundary the bulk copies accept (16 bytes) with room to spare.
size_t bg_half_floats(size_t n_pix) { return (n_pix * 3 + 63) / 64 * 64; }

psfs_status check_params(const psfs_params *p)
{
    if (!p) return fail(PSFS_ERR_INVALID_ARG, "params is NULL");
    const double v[5] = {p->p_detect, p->p_false_alarm, p->prior, p->threshold, p->log_fg_density};
    if (!finite_all(v, 5)) return fail(PSFS_ERR_INVALID_ARG, "params: non-finite value");
    if (p->p_detect < 0 || p->p_detect > 1) return fail(PSFS_ERR_INVALID_ARG, "p_detect outside [0, 1]");
    if (p->p_false_alarm < 0 || p->p_false_alarm > 1)
        return fail(PSFS_ERR_INVALID_ARG, "p_false_alarm outside [0, 1]");
    const double q = 0.5 * (p->p_detect + p->p_false_alarm);
    if (!(q > 0 && q < 1)) return fail(PSFS_ERR_INVALID_ARG, "(p_detect + p_false_alarm) / 2 must be in (0, 1)");
    if (!(p->prior > 0 && p->prior < 1)) return fail(PSFS_ERR_INVALID_ARG, "prior outside (0, 1)");
    if (!(p->threshold > 0 && p->threshold < 1)) return fail(PSFS_ERR_INVALID_ARG, "threshold outside (0, 1)");
    if (p->map_dtype != PSFS_MAP_F32 && p->map_dtype != PSFS_MAP_F16 && p->map_dtype != PSFS_MAP_BF16)
        return fail(PSFS_ERR_INVALID_ARG, "unknown map_dtype");
    return PSFS_OK;
}

void prof_free(psfs_handle *h);

void free_handle(psfs_handle *h)
{
    if (!h) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    cudaFree(h->maps);
    cudaFree(h->bg_mean);   // bg_hinv lives in the same allocation
    cudaFree(h->d_words);
    cudaFreeHost(h->h_words);
    cudaFree(h->tiles);
    cudaFree(h->tilecam);
    cudaFree(h->seq_tiles);
    cudaFree(h->seq_tilecam);
    cudaFree(h->st_images);
    cudaFree(h->st_occ);
    cudaFree(h->st_list);
    cudaFree(h->dl);
    cudaFree(h->dl_rec);
    cudaFree(h->dl_rec2);
    cudaFree(h->own_off);
    cudaFree(h->own_vox);
    cudaFree(h->own_cnt);
    cudaFree(h->own_sums);
    cudaFree(h->bw_tiles);
    cudaFree(h->bw_tilecam);
    cudaFree(h->bw_maps);
    cudaFree(h->maps2);
    cudaFree(h->gmaps[0]);
    cudaFree(h->gmaps[1]);
    cudaFree(h->surf_masks);
    for (int n = 0; n < 2; ++n) {
        if (h->io_stream[n]) cudaStreamSynchronize(h->io_stream[n]);
        if (h->io_stream[n]) cudaStreamDestroy(h->io_stream[n]);
    }
    for (int n = 0; n < kIoSlots; ++n) {
        for (cudaEvent_t e : {h->io_ev_in[n], h->io_ev_comp[n], h->io_ev_cnt[n], h->io_ev_out[n]})
            if (e) cudaEventDestroy(e);
        cudaFree(h->io_img[n]);
        cudaFree(h->io_occ[n]);
        cudaFree(h->io_list[n]);
        cudaFree(h->io_cnt[n]);
    }
    for (int n = 0; n < 2; ++n) {
        if (h->seq_stream[n]) cudaStreamSynchronize(h->seq_stream[n]);
        if (h->seq_stream[n]) cudaStreamDestroy(h->seq_stream[n]);
        if (h->seq_ev_map[n]) cudaEventDestroy(h->seq_ev_map[n]);
        if (h->seq_ev_fused[n]) cudaEventDestroy(h->seq_ev_fused[n]);
        if (h->seq_ev_done[n]) cudaEventDestroy(h->seq_ev_done[n]);
    }
    if (h->seq_ev_in) cudaEventDestroy(h->seq_ev_in);
    prof_free(h);
    cudaSetDevice(prev);
    delete h;
}

void prof_free(psfs_handle *h)
{
    for (cudaEvent_t e : h->prof_ev) cudaEventDestroy(e);
    h->prof_ev.clear();
    h->prof_stage.clear();
    h->prof_cap = 0;
    h->prof_n = 0;
}

// Brackets one launch with an event pair when tracing is on.
struct ProfScope {
    psfs_handle *h;
    cudaStream_t st;
    int slot = -1;
    ProfScope(psfs_handle *hh, int stage) : ProfScope(hh, stage, hh->stream) {}
    ProfScope(psfs_handle *hh, int stage, cudaStream_t s) : h(hh), st(s)
    {
        if (h->prof_cap > 0 && h->prof_n < h->prof_cap) {
            slot = h->prof_n++;
            h->prof_stage[slot] = stage;
            cudaEventRecord(h->prof_ev[2 * slot], st);
        }
    }
    ~ProfScope()
    {
        if (slot >= 0) cudaEventRecord(h->prof_ev[2 * slot + 1], st);
    }
};

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

psfs_status fill_fuse_args(psfs_handle *h, float *occ, uint32_t *list, uint32_t capacity,
                           uint32_t *count, FuseArgs *a)
{
    *a = h->fuse;
    a->occ = occ;
    a->list = list;
    a->capacity = capacity;
    a->count = count;
    a->occ_fstride = a->list_fstride = a->count_fstride = 0;
    return PSFS_OK;
}

psfs_status check_frame_outputs(const float *occupancy, const uint32_t *voxel_list, uint32_t capacity,
                                const uint32_t *count)
{
    if (!occupancy || !aligned(occupancy, 16)) return fail(PSFS_ERR_INVALID_ARG, "occupancy NULL or not 16-byte aligned");
    if (capacity > 0 && (!voxel_list || !aligned(voxel_list, 4)))
        return fail(PSFS_ERR_INVALID_ARG, "voxel_list NULL or not 4-byte aligned");
    if (!count || !aligned(count, 4)) return fail(PSFS_ERR_INVALID_ARG, "count NULL or not 4-byte aligned");
    return PSFS_OK;
}

// Tile shapes remembered by the autotuner, keyed by what the best shape
// depends on: grid size, camera count, image size and map type.
using TuneKey = std::tuple<int, int, int, int, int, int, int>;
struct Tuned {
    FuseShape shape;
    int seq_lk_ctas;
    int seq_group;
    bool seq_own;
    FuseShape seq_shape;
    int seq_rec;
};
std::mutex g_tune_mu;
std::map<TuneKey, Tuned> g_tuned;

TuneKey tune_key(const psfs_handle *h)
{
    return TuneKey(h->grid.nx, h->grid.ny, h->grid.nz, h->n_cams, h->W, h->H, h->params.map_dtype);
}

// (Re)plans the fuse kernel for `shape`: projection matrices, tile order and
// per (tile, camera) records, uploaded to freshly sized device arrays.
psfs_status replan(psfs_handle *h, const FuseShape &shape)
{
    std::vector<uint64_t> tiles;
    std::vector<int4> tilecam;
    FuseArgs f{};
    plan_fuse(h->grid, h->cams.data(), h->n_cams, h->params, shape, &f, &tiles, &tilecam);
    uint64_t *d_tiles = nullptr;
    int4 *d_tilecam = nullptr;
    if (cudaMalloc(&d_tiles, tiles.size() * sizeof(uint64_t)) != cudaSuccess ||
        cudaMalloc(&d_tilecam, tilecam.size() * sizeof(int4)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d_tiles);
        return fail(PSFS_ERR_NOMEM, "tile plan allocation");
    }
    cudaError_t e = cudaMemcpy(d_tiles, tiles.data(), tiles.size() * sizeof(uint64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(d_tilecam, tilecam.data(), tilecam.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d_tiles);
        cudaFree(d_tilecam);
        return fail_cuda(e, "tile plan upload");
    }
    cudaFree(h->tiles);
    cudaFree(h->tilecam);
    h->tiles = d_tiles;
    h->tilecam = d_tilecam;
    f.maps = h->maps;
    f.tiles = h->tiles;
    f.tilecam = h->tilecam;
    f.status = h->d_words;
    f.tmap_ok = h->tm_main_ok ? 1 : 0;
    for (int k = 0; k < kBoxClasses; ++k) f.tmap[k] = h->tm_main[k];
    h->fuse = f;
    h->n_tiles = f.n_tiles;
    h->shape = shape;
    return PSFS_OK;
}

// Plans the sequence path's own tile shape (a direct shape of the frame-group
// kernels) into seq_tiles / seq_tilecam.
psfs_status replan_seq(psfs_handle *h, const FuseShape &shape)
{
    std::vector<uint64_t> tiles;
    std::vector<int4> tilecam;
    FuseArgs f{};
    plan_fuse(h->grid, h->cams.data(), h->n_cams, h->params, shape, &f, &tiles, &tilecam);
    uint64_t *d_tiles = nullptr;
    int4 *d_tilecam = nullptr;
    if (cudaMalloc(&d_tiles, tiles.size() * sizeof(uint64_t)) != cudaSuccess ||
        cudaMalloc(&d_tilecam, tilecam.size() * sizeof(int4)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d_tiles);
        return fail(PSFS_ERR_NOMEM, "sequence tile plan allocation");
    }
    cudaError_t e = cudaMemcpy(d_tiles, tiles.data(), tiles.size() * sizeof(uint64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(d_tilecam, tilecam.data(), tilecam.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d_tiles);
        cudaFree(d_tilecam);
        return fail_cuda(e, "sequence tile plan upload");
    }
    cudaFree(h->seq_tiles);
    cudaFree(h->seq_tilecam);
    h->seq_tiles = d_tiles;
    h->seq_tilecam = d_tilecam;
    h->seq_n_tiles = f.n_tiles;
    h->seq_shape = shape;
    h->seq_own = true;
    return PSFS_OK;
}

// The tile shape of the sequence path.
const FuseShape &seq_shape_of(const psfs_handle *h) { return h->seq_own ? h->seq_shape : h->shape; }

}  // namespace

extern "C" {

const char *psfs_status_string(psfs_status s)
{
    switch (s) {
    case PSFS_OK: return "ok";
    case PSFS_ERR_INVALID_ARG: return "invalid argument";
    case PSFS_ERR_NOT_READY: return "background not set";
    case PSFS_ERR_CAPACITY: return "voxel list capacity exceeded";
    case PSFS_ERR_CUDA: return "CUDA error";
    case PSFS_ERR_TIMEOUT: return "device wait timed out";
    case PSFS_ERR_NOMEM: return "out of memory";
    case PSFS_ERR_BOUNDS: return "bounds check failed";
    }
    return "unknown status";
}

const char *psfs_last_error_message(void) { return psfs::last_failure(); }

void psfs_params_default(psfs_params *p)
{
    if (!p) return;
    p->p_detect = 0.9;
    p->p_false_alarm = 0.1;
    p->prior = 0.5;
    p->threshold = 0.5;
    p->log_fg_density = -3.0 * std::log(256.0);
    p->map_dtype = PSFS_MAP_F32;
}

psfs_status psfs_create(const psfs_grid *grid, const psfs_camera *cams, int32_t n_cams,
                        const psfs_params *params, void *stream, psfs_handle **out)
{
    if (!out) return fail(PSFS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!grid) return fail(PSFS_ERR_INVALID_ARG, "grid is NULL");
    if (!cams) return fail(PSFS_ERR_INVALID_ARG, "cams is NULL");
    if (n_cams < 1 || n_cams > PSFS_MAX_CAMS) return fail(PSFS_ERR_INVALID_ARG, "n_cams outside [1, PSFS_MAX_CAMS]");
    psfs_status st = check_params(params);
    if (st != PSFS_OK) return st;
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return fail(PSFS_ERR_INVALID_ARG, "grid size < 1");
    const uint64_t n_vox = (uint64_t)grid->nx * grid->ny * grid->nz;
    if (n_vox >= (1ull << 32)) return fail(PSFS_ERR_INVALID_ARG, "grid has 2^32 voxels or more");
    if (grid->nx > (1 << 24) || grid->ny > (1 << 24) || grid->nz > (1 << 24))
        return fail(PSFS_ERR_INVALID_ARG, "grid axis longer than 2^24");
    if (!finite_all(grid->origin, 3) || !std::isfinite(grid->voxel_size) || !(grid->voxel_size > 0))
        return fail(PSFS_ERR_INVALID_ARG, "grid origin / voxel_size not finite or voxel_size <= 0");
    const int W = cams[0].width, H = cams[0].height;
    if (W < 1 || H < 1 || W > 16384 || H > 16384) return fail(PSFS_ERR_INVALID_ARG, "camera size outside [1, 16384]");
    for (int c = 0; c < n_cams; ++c) {
        if (cams[c].width != W || cams[c].height != H)
            return fail(PSFS_ERR_INVALID_ARG, "cameras differ in width or height");
        if (!finite_all(cams[c].K, 9) || !finite_all(cams[c].R, 9) || !finite_all(cams[c].t, 3))
            return fail(PSFS_ERR_INVALID_ARG, "camera matrix not finite");
    }

    psfs_handle *h = new (std::nothrow) psfs_handle();
    if (!h) return fail(PSFS_ERR_NOMEM, "host allocation");
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        delete h;
        return fail_cuda(e, "cudaGetDevice");
    }
    h->stream = (cudaStream_t)stream;
    h->grid = *grid;
    h->cams.assign(cams, cams + n_cams);
    h->n_cams = n_cams;
    h->W = W;
    h->H = H;
    h->params = *params;
    h->n_pix = (int64_t)n_cams * W * H;
    h->map_elem = params->map_dtype == PSFS_MAP_F32 ? 4 : 2;

    // sensor constants of g(r)
    const double pd = params->p_detect, q = 0.5 * (params->p_detect + params->p_false_alarm);
    h->sc.pd = (float)pd;
    h->sc.one_minus_pd = (float)(1.0 - pd);
    h->sc.q = (float)q;
    h->sc.one_minus_q = (float)(1.0 - q);
    h->sc.a_zero_const_pos = (pd == 0.0);
    h->sc.a_zero_const_neg = (pd == 1.0);
    h->c0 = (float)(params->log_fg_density + 1.5 * std::log(M_PI));

    DeviceGuard guard(h->device);
    const size_t pix_bytes = (size_t)h->n_pix;
    if (cudaMalloc(&h->maps, pix_bytes * h->map_elem) != cudaSuccess ||
        cudaMalloc(&h->bg_mean, (bg_half_floats(pix_bytes) * 2) * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&h->d_words, 16 * sizeof(uint32_t)) != cudaSuccess ||
        cudaMallocHost(&h->h_words, 16 * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        free_handle(h);
        return fail(PSFS_ERR_NOMEM, "device scratch allocation");
    }
    h->bg_hinv = h->bg_mean + bg_half_floats(pix_bytes);
    h->tm_main_ok = encode_map_tensors(h->maps, params->map_dtype, W, H, n_cams, h->tm_main);
    e = cudaMemset(h->d_words, 0, 16 * sizeof(uint32_t));
    if (e != cudaSuccess) {
        free_handle(h);
        return fail_cuda(e, "psfs_create upload");
    }
    std::memset(h->h_words, 0, 16 * sizeof(uint32_t));

    // projection matrices, Morton tile order and per (tile, camera) records,
    // for the tile shape the autotuner chose for this kind of rig if any
    FuseShape shape = kDefaultFuseShape;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(tune_key(h));
        if (it != g_tuned.end()) {
            shape = it->second.shape;
            h->seq_lk_ctas = it->second.seq_lk_ctas;
            h->seq_group = it->second.seq_group;
            h->seq_own = it->second.seq_own;
            h->seq_shape = it->second.seq_shape;
            h->seq_rec = it->second.seq_rec;
        }
    }
    st = replan(h, shape);
    if (st == PSFS_OK && h->seq_own) st = replan_seq(h, h->seq_shape);
    if (st != PSFS_OK) {
        free_handle(h);
        return st;
    }
    *out = h;
    return PSFS_OK;
}

psfs_status psfs_set_background(psfs_handle *h, const float *mean, const float *var)
{
    if (!h) return fail(PSFS_ERR_INVALID_ARG, "handle is NULL");
    if (!mean || !var || !aligned(mean, 16) || !aligned(var, 16))
        return fail(PSFS_ERR_INVALID_ARG, "mean / var NULL or not 16-byte aligned");
    DeviceGuard guard(h->device);
    h->bg_ready = false;
    PSFS_CK(cudaMemsetAsync(h->d_words + 1, 0, sizeof(uint32_t), h->stream));
    PSFS_CK(launch_pack_background(mean, var, h->n_pix, h->bg_mean, h->bg_hinv, h->d_words + 1, h->stream));
    PSFS_CK(cudaMemcpyAsync(h->h_words + 1, h->d_words + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream));
    PSFS_CK(cudaStreamSynchronize(h->stream));
    if (h->h_words[1] != 0) return fail(PSFS_ERR_INVALID_ARG, "background: non-finite mean or variance outside [1e-6, 1e12]");
    h->bg_ready = true;
    return PSFS_OK;
}

static psfs_status enqueue_reconstruct(psfs_handle *h, const uint8_t *images, float *occupancy,
                                       uint32_t *voxel_list, uint32_t capacity, uint32_t *count)
{
    LikelihoodArgs la{};
    la.img = images;
    la.mean = h->bg_mean;
    la.hinv = h->bg_hinv;
    la.n_pix = h->n_pix;
    la.c0 = h->c0;
    la.sc = h->sc;
    la.out = h->maps;
    la.zero_word = count;
    la.status = h->d_words;
    {
        ProfScope ps(h, PSFS_STAGE_LIKELIHOOD);
        PSFS_CK(launch_likelihood(la, h->params.map_dtype, false, h->stream));
    }
    FuseArgs fa;
    fill_fuse_args(h, occupancy, voxel_list, capacity, count, &fa);
    {
        ProfScope ps(h, PSFS_STAGE_FUSE);
        PSFS_CK(launch_fuse(fa, h->shape, h->params.map_dtype, h->stream));
    }
    return PSFS_OK;
}

psfs_status psfs_reconstruct(psfs_handle *h, const uint8_t *images, float *occupancy,
                             uint32_t *voxel_list, uint32_t capacity, uint32_t *count)
{
    if (!h) return fail(PSFS_ERR_INVALID_ARG, "handle is NULL");
    if (!images || !aligned(images, 16)) return fail(PSFS_ERR_INVALID_ARG, "images NULL or not 16-byte aligned");
    psfs_status st = check_frame_outputs(occupancy, voxel_list, capacity, count);
    if (st != PSFS_OK) return st;
    if (!h->bg_ready) return fail(PSFS_ERR_NOT_READY, "psfs_set_background has not succeeded");
    DeviceGuard guard(h->device);
    return enqueue_reconstruct(h, images, occupancy, voxel_list, capacity, count);
}

// L2 residency of the packed background on the likelihood stream of the
// sequence path: the background is the same every frame (59 MB at
// 8 x 640 x 480) and fits the persisting part of the 126 MB L2, so frames
// after the first read it from L2 instead of HBM.
static psfs_status apply_l2_window(psfs_handle *h)
{
    if (!h->seq_stream[0]) return PSFS_OK;
    cudaStreamAttrValue v;
    std::memset(&v, 0, sizeof(v));
    if (h->bg_l2) {
        int max_win = 0, max_persist = 0;
        PSFS_CK(cudaDeviceGetAttribute(&max_win, cudaDevAttrMaxAccessPolicyWindowSize, h->device));
        PSFS_CK(cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, h->device));
        const size_t bytes = bg_half_floats((size_t)h->n_pix) * 2 * sizeof(float);
        size_t limit = 0;
        PSFS_CK(cudaDeviceGetLimit(&limit, cudaLimitPersistingL2CacheSize));
        const size_t want = std::min(bytes, (size_t)max_persist);
        if (limit < want) PSFS_CK(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want));
        v.accessPolicyWindow.base_ptr = h->bg_mean;
        v.accessPolicyWindow.num_bytes = std::min(bytes, (size_t)max_win);
        v.accessPolicyWindow.hitRatio = std::min(1.0f, (float)want / (float)v.accessPolicyWindow.num_bytes);
        v.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        v.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    }
    PSFS_CK(cudaStreamSetAttribute(h->seq_stream[0], cudaStreamAttributeAccessPolicyWindow, &v));
    return PSFS_OK;
}

static psfs_status seq_setup(psfs_handle *h)
{
    if (h->seq_stream[0]) return PSFS_OK;
    if (cudaMalloc(&h->maps2, (size_t)h->n_pix * h->map_elem) != cudaSuccess) {
        cudaGetLastError();
        return fail(PSFS_ERR_NOMEM, "second map buffer");
    }
    h->tm_alt_ok = encode_map_tensors(h->maps2, h->params.map_dtype, h->W, h->H, h->n_cams, h->tm_alt);
    for (int n = 0; n < 2; ++n) {
        PSFS_CK(cudaStreamCreateWithFlags(&h->seq_stream[n], cudaStreamNonBlocking));
        PSFS_CK(cudaEventCreateWithFlags(&h->seq_ev_map[n], cudaEventDisableTiming));
        PSFS_CK(cudaEventCreateWithFlags(&h->seq_ev_fused[n], cudaEventDisableTiming));
        PSFS_CK(cudaEventCreateWithFlags(&h->seq_ev_done[n], cudaEventDisableTiming));
    }
    PSFS_CK(cudaEventCreateWithFlags(&h->seq_ev_in, cudaEventDisableTiming));
    return apply_l2_window(h);
}

// Group map buffers for `frames` frames per group (waits for the sequence
// streams before it replaces smaller ones).
static psfs_status ensure_group_maps(psfs_handle *h, int frames)
{
    if (frames <= h->group_cap) return PSFS_OK;
    PSFS_CK(cudaStreamSynchronize(h->seq_stream[0]));
    PSFS_CK(cudaStreamSynchronize(h->seq_stream[1]));
    for (int b = 0; b < 2; ++b) {
        cudaFree(h->gmaps[b]);
        h->gmaps[b] = nullptr;
    }
    h->group_cap = 0;
    for (int b = 0; b < 2; ++b) {
        if (cudaMalloc(&h->gmaps[b], (size_t)h->n_pix * frames * h->map_elem) != cudaSuccess) {
            cudaGetLastError();
            return fail(PSFS_ERR_NOMEM, "frame-group map buffers");
        }
    }
    h->group_cap = frames;
    return PSFS_OK;
}

// Frames in the next unit of a sequence: the largest group size that fits the
// remaining frames (group, group / 2, ... down to 2 frames, each with the
// tile shape), else one frame.  (Starting with smaller units to shorten the
// first likelihood pass, which nothing overlaps, measured slower: smaller
// groups cost more per frame in the likelihood.)
static int unit_frames(const psfs_handle *h, int group, int remaining)
{
    for (int g = group; g >= 2; g >>= 1)
        if (g <= remaining && group_shape_supported(seq_shape_of(h), g, (int)h->map_elem, h->seq_rec)) return g;
    return 1;
}

// Enqueues n_frames frames with the given element strides between frames
// (a stride of 0 repeats the same buffer, which only the autotuner does when
// it has no room for copies of its frame).
// Frames go in units (unit_frames): groups of `group` frames (one likelihood
// launch and one fusion launch per plane of pixel records) while whole groups
// remain, then the largest smaller groups that fit, then single frames.  Unit u's likelihood (stream 0)
// writes map buffer u & 1 while the fusion of unit u - 1 (stream 1) reads the
// other one.
static psfs_status enqueue_sequence(psfs_handle *h, int32_t n_frames, const uint8_t *images, size_t img_stride,
                                    float *occupancy, size_t occ_stride, uint32_t *voxel_lists,
                                    size_t list_stride, uint32_t capacity, uint32_t *counts, size_t count_stride,
                                    int lk_ctas, int group)
{
    psfs_status st = seq_setup(h);
    if (st != PSFS_OK) return st;
    const FuseShape sshape = seq_shape_of(h);
    if (group > 1 && !group_shape_supported(sshape, group, (int)h->map_elem, h->seq_rec)) group = 1;
    const int first_unit = unit_frames(h, group, n_frames);   // the largest
    if (first_unit > 1) {
        st = ensure_group_maps(h, first_unit);
        if (st != PSFS_OK) return st;
    }
    cudaStream_t sl = h->seq_stream[0], sf = h->seq_stream[1];
    void *bufs[2] = {h->maps, h->maps2};
    PSFS_CK(cudaEventRecord(h->seq_ev_in, h->stream));
    PSFS_CK(cudaStreamWaitEvent(sl, h->seq_ev_in, 0));
    PSFS_CK(cudaStreamWaitEvent(sf, h->seq_ev_in, 0));
    int f = 0;
    for (int u = 0; f < n_frames; ++u) {
        const int nf = unit_frames(h, group, n_frames - f);
        const int b = u & 1;
        if (u >= 2) PSFS_CK(cudaStreamWaitEvent(sl, h->seq_ev_fused[b], 0));   // unit u-2 done with buffer b
        void *buf = nf > 1 ? h->gmaps[b] : bufs[b];
        LikelihoodArgs la{};
        la.img = images + (size_t)f * img_stride;
        la.mean = h->bg_mean;
        la.hinv = h->bg_hinv;
        la.n_pix = h->n_pix;
        la.c0 = h->c0;
        la.sc = h->sc;
        la.out = buf;
        la.zero_word = counts + (size_t)f * count_stride;
        la.status = h->d_words;
        la.img_fstride = (int64_t)img_stride;
        la.zero_fstride = (int64_t)count_stride;
        {
            ProfScope ps(h, PSFS_STAGE_LIKELIHOOD, sl);
            if (nf > 1)
                PSFS_CK(launch_likelihood_group(la, nf, h->params.map_dtype, sl, lk_ctas, h->seq_rec));
            else
                PSFS_CK(launch_likelihood(la, h->params.map_dtype, false, sl, lk_ctas));
        }
        PSFS_CK(cudaEventRecord(h->seq_ev_map[b], sl));
        PSFS_CK(cudaStreamWaitEvent(sf, h->seq_ev_map[b], 0));
        FuseArgs fa;
        fill_fuse_args(h, occupancy + (size_t)f * occ_stride, voxel_lists + (size_t)f * list_stride, capacity,
                       counts + (size_t)f * count_stride, &fa);
        fa.maps = buf;
        if (h->seq_own) {   // the sequence path's own tile plan
            fa.tiles = h->seq_tiles;
            fa.tilecam = h->seq_tilecam;
            fa.n_tiles = h->seq_n_tiles;
        }
        if (nf > 1) {
            fa.tmap_ok = 0;
            fa.occ_fstride = (int64_t)occ_stride;
            fa.list_fstride = (int64_t)list_stride;
            fa.count_fstride = (int64_t)count_stride;
        } else if (b == 1) {
            fa.tmap_ok = h->tm_alt_ok ? 1 : 0;
            for (int k = 0; k < kBoxClasses; ++k) fa.tmap[k] = h->tm_alt[k];
        }
        {
            ProfScope ps(h, PSFS_STAGE_FUSE, sf);
            if (nf > 1) {
                PSFS_CK(launch_fuse_group(fa, sshape, nf, h->params.map_dtype, sf, h->seq_rec));
            } else {
                PSFS_CK(launch_fuse(fa, sshape, h->params.map_dtype, sf));
            }
        }
        PSFS_CK(cudaEventRecord(h->seq_ev_fused[b], sf));
        f += nf;
    }
    PSFS_CK(cudaEventRecord(h->seq_ev_done[0], sl));
    PSFS_CK(cudaEventRecord(h->seq_ev_done[1], sf));
    PSFS_CK(cudaStreamWaitEvent(h->stream, h->seq_ev_done[0], 0));
    PSFS_CK(cudaStreamWaitEvent(h->stream, h->seq_ev_done[1], 0));
    return PSFS_OK;
}

psfs_status psfs_set_background_l2(psfs_handle *h, int32_t enable)
{
    if (!h) return fail(PSFS_ERR_INVALID_ARG, "handle is NULL");
    DeviceGuard guard(h->device);
    h->bg_l2 = enable != 0;
    psfs_status st = seq_setup(h);
    if (st != PSFS_OK) return st;
    return apply_l2_window(h);
}

psfs_status psfs_reconstruct_sequence(psfs_handle *h, int32_t n_frames, const uint8_t *images,
                                      float *occupancy, uint32_t *voxel_lists, uint32_t capacity,
                                      uint32_t *counts)
{
    if (!h) return fail(PSFS_ERR_INVALID_ARG, "handle is NULL");
    if (n_frames < 0) return fail(PSFS_ERR_INVALID_ARG, "n_frames < 0");
    if (n_frames == 0) return PSFS_OK;
    if (!images || !aligned(images, 16)) return fail(PSFS_ERR_INVALID_ARG, "images NULL or not 16-byte aligned");
    if ((h->n_pix * 3) % 16 != 0) return fail(PSFS_ERR_INVALID_ARG, "frame size not a multiple of 16 bytes");
    const uint64_t n_vox = (uint64_t)h->grid.nx * h->grid.ny * h->grid.nz;
    if (n_vox % 4 != 0) return fail(PSFS_ERR_INVALID_ARG, "voxel count not a multiple of 4");
    psfs_status st = check_frame_outputs(occupancy, voxel_lists, capacity, counts);
    if (st != PSFS_OK) return st;
    DeviceGuard guard(h->device);
    if (!h->bg_ready) return fail(PSFS_ERR_NOT_READY, "psfs_set_background has not succeeded");
    return enqueue_sequence(h, n_frames, images, (size_t)h->n_pix * 3, occupancy, n_vox, voxel_lists, capacity,
                            capacity, counts, 1, h->seq_lk_ctas, h->seq_group);
}

// Staging of the host-buffer sequence path: kIoSlots slots of `frames` frames.
static psfs_status io_setup(psfs_handle *h, int frames, uint32_t capacity)
{
    if (!h->io_stream[0]) {
        for (int n = 0; n < 2; ++n) PSFS_CK(cudaStreamCreateWithFlags(&h->io_stream[n], cudaStreamNonBlocking));
        for (int n = 0; n < kIoSlots; ++n) {
            PSFS_CK(cudaEventCreateWithFlags(&h->io_ev_in[n], cudaEventDisableTiming));
            PSFS_CK(cudaEventCreateWithFlags(&h->io_ev_comp[n], cudaEventDisableTiming));
            PSFS_CK(cudaEventCreateWithFlags(&h->io_ev_cnt[n], cudaEventDisableTiming));
            PSFS_CK(cudaEventCreateWithFlags(&h->io_ev_out[n], cudaEventDisableTiming));
        }
    }
    if (frames <= h->io_frames && capacity <= h->io_cap) return PSFS_OK;
    PSFS_CK(cudaStreamSynchronize(h->io_stream[0]));
    PSFS_CK(cudaStreamSynchronize(h->io_stream[1]));
    PSFS_CK(cudaStreamSynchronize(h->stream));
    const uint64_t n_vox = (uint64_t)h->grid.nx * h->grid.ny * h->grid.nz;
    frames = std::max(frames, h->io_frames);
    capacity = std::max(capacity, h->io_cap);
    h->io_frames = 0;
    h->io_cap = 0;
    for (int n = 0; n < kIoSlots; ++n) {
        cudaFree(h->io_img[n]);
        cudaFree(h->io_occ[n]);
        cudaFree(h->io_list[n]);
        cudaFree(h->io_cnt[n]);
        h->io_img[n] = nullptr;
        h->io_occ[n] = nullptr;
        h->io_list[n] = nullptr;
        h->io_cnt[n] = nullptr;
    }
    for (int n = 0; n < kIoSlots; ++n) {
        if (cudaMalloc(&h->io_img[n], (size_t)frames * h->n_pix * 3) != cudaSuccess ||
            cudaMalloc(&h->io_occ[n], (size_t)frames * n_vox * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&h->io_list[n], (size_t)frames * std::max<uint32_t>(capacity, 1) * sizeof(uint32_t)) !=
                cudaSuccess ||
            cudaMalloc(&h->io_cnt[n], (size_t)frames * sizeof(uint32_t)) != cudaSuccess) {
            cudaGetLastError();
            return fail(PSFS_ERR_NOMEM, "host-buffer sequence staging");
        }
    }
    h->io_frames = frames;
    h->io_cap = capacity;
    return PSFS_OK;
}

psfs_status psfs_reconstruct_sequence_host(psfs_handle *h, int32_t n_frames, const uint8_t *h_images,
                                           float *h_occupancy, uint32_t *h_lists, uint32_t capacity,
                                           uint32_t *h_counts)
{
    if (!h) return fail(PSFS_ERR_INVALID_ARG, "handle is NULL");
    if (n_frames < 0) return fail(PSFS_ERR_INVALID_ARG, "n_frames < 0");
    if (n_frames == 0) return PSFS_OK;
    if (!h_images) return fail(PSFS_ERR_INVALID_ARG, "h_images is NULL");
    if (capacity > 0 && !h_lists) return fail(PSFS_ERR_INVALID_ARG, "h_lists is NULL");
    if (!h_counts) return fail(PSFS_ERR_INVALID_ARG, "h_counts is NULL");
    if ((h->n_pix * 3) % 16 != 0) return fail(PSFS_ERR_INVALID_ARG, "frame size not a multiple of 16 bytes");
    const uint64_t n_vox = (uint64_t)h->grid.nx * h->grid.ny * h->grid.nz;
    if (n_vox % 4 != 0) return fail(PSFS_ERR_INVALID_ARG, "voxel count not a multiple of 4");
    if (!h->bg_ready) return fail(PSFS_ERR_NOT_READY, "psfs_set_background has not succeeded");
    DeviceGuard guard(h->device);
    // chunks of 4 frames per slot: the copies of one chunk overlap the
    // kernels of the next.  The host link (about 200 GB/s each way) is slower
    // than the kernels by several times, so the chunk size is set by the
    // copies: at 128^3 x 8 x 640 x 480 chunks of 4 frames took 5.49 ms per
    // 100 frames with the grids copied out, against 5.52-5.57 for 3, 5 or 6
    // frames, 5.66 for 8 and 6.45 for 1 (the counts and lists alone: 3.66
    // ms for 4 or 8 frames).
    const int chunk = std::min<int>(n_frames, 4);
    psfs_status st = io_setup(h, chunk, capacity);
    if (st != PSFS_OK) return st;
    const size_t frame_bytes = (size_t)h->n_pix * 3;
    const uint32_t lcap = std::max<uint32_t>(capacity, 1);
    cudaStream_t cin = h->io_stream[0], cout = h->io_stream[1];
    PSFS_CK(cudaEventRecord(h->io_ev_in[0], h->stream));   // after earlier work on the handle
    PSFS_CK(cudaStreamWaitEvent(cin, h->io_ev_in[0], 0));
    const int n_chunks = (n_frames + chunk - 1) / chunk;
    bool overflow = false;
    // list entries of chunk p go out once its counts are on the host
    auto drain_lists = [&](int p) -> psfs_status {
        const int q = p % kIoSlots, f0 = p * chunk, nf = std::min(chunk, n_frames - f0);
        PSFS_CK(cudaEventSynchronize(h->io_ev_cnt[q]));
        for (int f = 0; f < nf; ++f) {
            const uint32_t n = h_counts[f0 + f];
            overflow |= n > capacity;
            const uint32_t m = std::min(n, capacity);
            if (m)
                PSFS_CK(cudaMemcpyAsync(h_lists + (size_t)(f0 + f) * capacity, h->io_list[q] + (size_t)f * lcap,
                                        (size_t)m * sizeof(uint32_t), cudaMemcpyDeviceToHost, cout));
        }
        PSFS_CK(cudaEventRecord(h->io_ev_out[q], cout));
        return PSFS_OK;
    };
    // slot q = k mod 3: the copy in of chunk k waits until chunk k - 3's
    // kernels have read the images of slot q; chunk k's kernels wait until
    // chunk k - 3's results have been copied out of slot q.  The list copies
    // of chunk k - 2 are enqueued (once its counts are on the host, which
    // they are by then unless the copies out lag two chunks behind) before
    // the copies out of chunk k, so copies in, kernels and copies out of
    // consecutive chunks overlap and the host rarely waits.
    constexpr int kLag = kIoSlots - 1;
    for (int k = 0; k < n_chunks && st == PSFS_OK; ++k) {
        const int q = k % kIoSlots, f0 = k * chunk, nf = std::min(chunk, n_frames - f0);
        if (k >= kIoSlots) PSFS_CK(cudaStreamWaitEvent(cin, h->io_ev_comp[q], 0));
        PSFS_CK(cudaMemcpyAsync(h->io_img[q], h_images + (size_t)f0 * frame_bytes, (size_t)nf * frame_bytes,
                                cudaMemcpyHostToDevice, cin));
        PSFS_CK(cudaEventRecord(h->io_ev_in[q], cin));
        PSFS_CK(cudaStreamWaitEvent(h->stream, h->io_ev_in[q], 0));
        if (k >= kIoSlots) PSFS_CK(cudaStreamWaitEvent(h->stream, h->io_ev_out[q], 0));
        st = enqueue_sequence(h, nf, h->io_img[q], frame_bytes, h->io_occ[q], n_vox, h->io_list[q], lcap, capacity,
                              h->io_cnt[q], 1, h->seq_lk_ctas, h->seq_group);
        if (st != PSFS_OK) break;
        PSFS_CK(cudaEventRecord(h->io_ev_comp[q], h->stream));
        if (k >= kLag) {
            st = drain_lists(k - kLag);
            if (st != PSFS_OK) break;
        }
        PSFS_CK(cudaStreamWaitEvent(cout, h->io_ev_comp[q], 0));
        PSFS_CK(cudaMemcpyAsync(h_counts + f0, h->io_cnt[q], (size_t)nf * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                cout));
        PSFS_CK(cudaEventRecord(h->io_ev_cnt[q], cout));
        if (h_occupancy)
            PSFS_CK(cudaMemcpyAsync(h_occupancy + (size_t)f0 * n_vox, h->io_occ[q], (size_t)nf * n_vox * sizeof(float),
                                    cudaMemcpyDeviceToHost, cout));
    }
    for (int p = std::max(0, n_chunks - kLag); p < n_chunks && st == PSFS_OK; ++p) st = drain_lists(p);
    PSFS_CK(cudaStreamSynchronize(cout));
    PSFS_CK(cudaStreamSynchronize(h->stream));
    if (st != PSFS_OK) return st;
    if (overflow) {
        // the capacity bit was set by these frames: clear it here
        PSFS_CK(cudaMemsetAsync(h->d_words, 0, sizeof(uint32_t), h->stream));
        PSFS_CK(cudaStreamSynchronize(h->stream));
        return fail(PSFS_ERR_CAPACITY, "voxel list capacity exceeded");
    }
    return PSFS_OK;
}

psfs_status psfs_particle_weights(psfs_handle *h, int32_t n_particles, int32_t n_cyl, const float *cylinders,
                                  int32_t kt, int32_t kw, const uint8_t *masks, float *weights, float *terms)
{
    if (!h) return fail(PSFS_ERR_INVALID_ARG, "handle is NULL");
    if (n_particles < 0) return fail(PSFS_ERR_INVALID_ARG, "n_particles < 0");
    if (n_particles == 0) return PSFS_OK;
    if (n_cyl < 1 || n_cyl > 64) return fail(PSFS_ERR_INVALID_ARG, "n_cyl outside [1, 64]");
    if (kt < 1 || kt > 64 || kw < 1 || kw > 64) return fail(PSFS_ERR_INVALID_ARG, "kt or kw outside [1, 64]");
    if (!cylinders || !aligned(cylinders, 4)) return fail(PSFS_ERR_INVALID_ARG, "cylinders NULL or misaligned");
    if (!masks) return fail(PSFS_ERR_INVALID_ARG, "masks is NULL");
    if (!weights || !aligned(weights, 4)) return fail(PSFS_ERR_INVALID_ARG, "weights NULL or misaligned");
    if (terms && !aligned(terms, 4)) return fail(PSFS_ERR_INVALID_ARG, "terms misaligned");
    DeviceGuard guard(h->device);
    WeightArgs a{};
    for (int c = 0; c < h->n_cams; ++c) {
        const psfs_camera &cam = h->cams[c];
        for (int r = 0; r < 3; ++r) {
            for (int col = 0; col < 3; ++col) {
                double v = 0.0;
                for (int q = 0; q < 3; ++q) v += cam.K[3 * r + q] * cam.R[3 * q + col];
                a.P[c][4 * r + col] = (float)v;
            }
            double v = 0.0;
            for (int q = 0; q < 3; ++q) v += cam.K[3 * r + q] * cam.t[q];
            a.P[c][4 * r + 3] = (float)v;
            double C = 0.0;
            for (int q = 0; q < 3; ++q) C -= cam.R[3 * q + r] * cam.t[q];
            a.C[c][r] = (float)C;
        }
    }
    a.n_cams = h->n_cams;
    a.W = h->W;
    a.H = h->H;
    a.n_cyl = n_cyl;
    a.kt = kt;
    a.kw = kw;
    a.cyl = cylinders;
    a.masks = masks;
    a.weights = weights;
    a.terms = terms;
    PSFS_CK(launch_weights(a, n_particles, h->stream));
    return PSFS_OK;
}

psfs_status psfs_reproject(psfs_handle *h, int32_t n_frames, const uint32_t *voxel_lists, uint32_t list_stride,
                           const uint32_t *counts, uint8_t *masks)
{
    if (!h) return fail(PSFS_ERR_INVALID_ARG, "handle is NULL");
    if (n_frames < 0) return fail(PSFS_ERR_INVALID_ARG, "n_frames < 0");
    if (n_frames == 0) return PSFS_OK;
    if (list_stride > 0 && (!voxel_lists || !aligned(voxel_lists, 4)))
        return fail(PSFS_ERR_INVALID_ARG, "voxel_lists NULL or not 4-byte aligned");
    if (!counts || !aligned(counts, 4)) return fail(PSFS_ERR_INVALID_ARG, "counts NULL or not 4-byte aligned");
    if (!masks) return fail(PSFS_ERR_INVALID_ARG, "masks is NULL");
    if (n_frames > 65535) return fail(PSFS_ERR_INVALID_ARG, "more than 65535 frames in one call");
    DeviceGuard guard(h->device);
    ReprojectArgs a{};
    for (int c = 0; c < h->n_cams; ++c) a.cam[c] = h->fuse.cam[c];
    plan_pixel_rays(h->grid, h->cams.data(), h->n_cams, h->fuse, a.inv);
    a.lists = voxel_lists;
    a.list_stride = list_stride;
    a.counts = counts;
    a.masks = masks;
    a.n_cams = h->n_cams;
    a.W = h->W;
    a.H = h->H;
    a.nx = h->grid.nx;
    a.ny = h->grid.ny;
    a.nz = h->grid.nz;
    a.ci = h->fuse.ci;
    a.cj = h->fuse.cj;
    a.ck = h->fuse.ck;
    a.n_vox = (uint32_t)((uint64_t)h->grid.nx * h->grid.ny * h->grid.nz);
    a.status = h->d_words;
    ProfScope ps(h, PSFS_STAGE_REPROJECT);
    PSFS_CK(launch_reproject(a, n_frames, h->stream));
    return PSFS_OK;
}

psfs_status psfs_smooth(psfs_handle *h, int32_t n_frames, const float *occupancy, float *smoothed,
                        uint32_t *voxel_lists, uint32_t capacity, uint32_t *counts)
{
    if (!h) return fail(PSFS_ERR_INVALID_ARG, "handle is NULL");
    if (n_frames < 0) return fail(PSFS_ERR_INVALID_ARG, "n_frames < 0");
    if (n_frames == 0) return PSFS_OK;
    if (!occupancy || !aligned(occupancy, 4)) return fail(PSFS_ERR_INVALID_ARG, "occupancy NULL or not 4-byte aligned");
    if (smoothed && !aligned(smoothed, 4)) return fail(PSFS_ERR_INVALID_ARG, "smoothed not 4-byte aligned");
    if (capacity > 0 && (!voxel_lists || !aligned(voxel_lists, 4)))
        return fail(PSFS_ERR_INVALID_ARG, "voxel_lists NULL or not 4-byte aligned");
    if (!counts || !aligned(counts, 4)) return fail(PSFS_ERR_INVALID_ARG, "counts NULL or not 4-byte aligned");
    const int tz = (h->grid.nz + 31) / 32;   // z-tiles of 32 planes per frame
    if ((int64_t)tz * n_frames > 65535) return fail(PSFS_ERR_INVALID_ARG, "too many frames for one call");
    DeviceGuard guard(h->device);
    SmoothArgs a{};
    a.prob = occupancy;
    a.smoothed = smoothed;
    a.lists = voxel_lists;
    a.capacity = capacity;
    a.counts = counts;
    a.nx = h->grid.nx;
    a.ny = h->grid.ny;
    a.nz = h->grid.nz;
    a.threshold = (float)h->params.threshold;
    a.status = h->d_words;
    ProfScope ps(h, PSFS_STAGE_SMOOTH);
    PSFS_CK(launch_smooth(a, n_frames, h->stream));
    return PSFS_OK;
}

psfs_status psfs_surface(psfs_handle *h, int32_t n_frames, const uint32_t *voxel_lists, uint32_t list_stride,
                         const uint32_t *counts, uint32_t *surface_lists, uint32_t surface_capacity,
                         uint32_t *surface_counts)
{
    if (!h) return fail(PSFS_ERR_INVALID_ARG, "handle is NULL");
    if (n_frames < 0) return fail(PSFS_ERR_INVALID_ARG, "n_frames < 0");
    if (n_frames == 0) return PSFS_OK;
    if (list_stride > 0 && (!voxel_lists || !aligned(voxel_lists, 4)))
        return fail(PSFS_ERR_INVALID_ARG, "voxel_lists NULL or not 4-byte aligned");
    if (!counts || !aligned(counts, 4)) return fail(PSFS_ERR_INVALID_ARG, "counts NULL or not 4-byte aligned");
    if (surface_capacity > 0 && (!surface_lists || !aligned(surface_lists, 4)))
        return fail(PSFS_ERR_INVALID_ARG, "surface_lists NULL or not 4-byte aligned");
    if (!surface_counts || !aligned(surface_counts, 4))
        return fail(PSFS_ERR_INVALID_ARG, "surface_counts NULL or not 4-byte aligned");
    DeviceGuard guard(h->device);
    const uint64_t n_vox = (uint64_t)h->grid.nx * h->grid.ny * h->grid.nz;
    const uint32_t words = (uint32_t)((n_vox + 31) / 32);
    if (n_frames > h->surf_frames) {
        PSFS_CK(cudaStreamSynchronize(h->stream));
        cudaFree(h->surf_masks);
        h->surf_masks = nullptr;
        h->surf_frames = 0;
        if (cudaMalloc(&h->surf_masks, (size_t)n_frames * words * sizeof(uint32_t)) != cudaSuccess) {
            cudaGetLastError();
            return fail(PSFS_ERR_NOMEM, "surface bitmasks");
        }
        h->surf_frames = n_frames;
    }
    SurfaceArgs a{};
    a.lists = voxel_lists;
    a.list_stride = list_stride;
    a.counts = counts;
    a.surface_lists = surface_lists;
    a.surface_capacity = surface_capacity;
    a.surface_counts = surface_counts;
    a.masks = h->surf_masks;
    a.mask_words = words;
    a.n_vox = (uint32_t)n_vox;
    a.nx = h->grid.nx;
    a.ny = h->grid.ny;
    a.nz = h->grid.nz;
    a.status = h->d_words;
    ProfScope ps(h, PSFS_STAGE_SURFACE);
    PSFS_CK(launch_surface(a, n_frames, h->stream));
    return PSFS_OK;
}

psfs_status psfs_reconstruct_host(psfs_handle *h, const uint8_t *h_images, float *h_occupancy,
                                  uint32_t *h_list, uint32_t capacity, uint32_t *h_count)
{
    if (!h) return fail(PSFS_ERR_INVALID_ARG, "handle is NULL");
    if (!h_images) return fail(PSFS_ERR_INVALID_ARG, "h_images is NULL");
    if (capacity > 0 && !h_list) return fail(PSFS_ERR_INVALID_ARG, "h_list is NULL");
    if (!h_count) return fail(PSFS_ERR_INVALID_ARG, "h_count is NULL");
    if (!h->bg_ready) return fail(PSFS_ERR_NOT_READY, "psfs_set_background has not succeeded");
    DeviceGuard guard(h->device);
    const uint64_t n_vox = (uint64_t)h->grid.nx * h->grid.ny * h->grid.nz;
    if (!h->st_images) {
        if (cudaMalloc(&h->st_images, (size_t)h->n_pix * 3) != cudaSuccess ||
            cudaMalloc(&h->st_occ, n_vox * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return fail(PSFS_ERR_NOMEM, "host-path staging allocation");
        }
    }
    if (capacity > h->st_list_cap) {
        cudaFree(h->st_list);
        h->st_list = nullptr;
        h->st_list_cap = 0;
        if (cudaMalloc(&h->st_list, (size_t)capacity * sizeof(uint32_t)) != cudaSuccess) {
            cudaGetLastError();
            return fail(PSFS_ERR_NOMEM, "host-path list allocation");
        }
        h->st_list_cap = capacity;
    }
    PSFS_CK(cudaMemcpyAsync(h->st_images, h_images, (size_t)h->n_pix * 3, cudaMemcpyHostToDevice, h->stream));
    psfs_status st = enqueue_reconstruct(h, h->st_images, h->st_occ, h->st_list, capacity, h->d_words + 2);
    if (st != PSFS_OK) return st;
    if (h_occupancy)
        PSFS_CK(cudaMemcpyAsync(h_occupancy, h->st_occ, n_vox * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    PSFS_CK(cudaMemcpyAsync(h->h_words + 2, h->d_words + 2, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream));
    PSFS_CK(cudaStreamSynchronize(h->stream));
    const uint32_t n = h->h_words[2];
    *h_count = n;
    const uint32_t ncopy = std::min(n, capacity);
    if (ncopy) {
        PSFS_CK(cudaMemcpyAsync(h_list, h->st_list, (size_t)ncopy * sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream));
        PSFS_CK(cudaStreamSynchronize(h->stream));
    }
    // the capacity bit may have been set by this frame: clear it here
    PSFS_CK(cudaMemsetAsync(h->d_words, 0, sizeof(uint32_t), h->stream));
    if (n > capacity) return fail(PSFS_ERR_CAPACITY, "voxel list capacity exceeded");
    return PSFS_OK;
}

psfs_status psfs_fuse_slm(psfs_handle *h, const float *slm, float *occupancy, uint32_t *voxel_list,
                          uint32_t capacity, uint32_t *count)
{
    if (!h) return fail(PSFS_ERR_INVALID_ARG, "handle is NULL");
    if (!slm || !aligned(slm, 16)) return fail(PSFS_ERR_INVALID_ARG, "slm NULL or not 16-byte aligned");
    psfs_status st = check_frame_outputs(occupancy, voxel_list, capacity, count);
    if (st != PSFS_OK) return st;
    DeviceGuard guard(h->device);
    const double pd = h->params.p_detect, q = 0.5 * (h->params.p_detect + h->params.p_false_alarm);
    SlmToMapArgs sa{};
    sa.slm = slm;
    sa.n_pix = h->n_pix;
    sa.da = (float)(2.0 * pd - 1.0);
    sa.one_minus_pd = (float)(1.0 - pd);
    sa.db = (float)(2.0 * q - 1.0);
    sa.one_minus_q = (float)(1.0 - q);
    sa.out = h->maps;
    sa.zero_word = count;
    {
        ProfScope ps(h, PSFS_STAGE_LIKELIHOOD);
        PSFS_CK(launch_slm_to_map(sa, h->params.map_dtype, h->stream));
    }
    FuseArgs fa;
    fill_fuse_args(h, occupancy, voxel_list, capacity, count, &fa);
    {
        ProfScope ps(h, PSFS_STAGE_FUSE);
        PSFS_CK(launch_fuse(fa, h->shape, h->params.map_dtype, h->stream));
    }
    return PSFS_OK;
}

psfs_status psfs_get_likelihood(psfs_handle *h, const uint8_t *images, float *slm_out)
{
    if (!h) return fail(PSFS_ERR_INVALID_ARG, "handle is NULL");
    if (!images || !aligned(images, 16)) return fail(PSFS_ERR_INVALID_ARG, "images NULL or not 16-byte aligned");
    if (!slm_out || !aligned(slm_out, 16)) return fail(PSFS_ERR_INVALID_ARG, "slm_out NULL or not 16-byte aligned");
    if (!h->bg_ready) return fail(PSFS_ERR_NOT_READY, "psfs_set_background has not succeeded");
    DeviceGuard guard(h->device);
    LikelihoodArgs la{};
    la.img = images;
    la.mean = h->bg_mean;
    la.hinv = h->bg_hinv;
    la.n_pix = h->n_pix;
    la.c0 = h->c0;
    la.sc = h->sc;
    la.out = slm_out;
    la.zero_word = nullptr;
    la.status = h->d_words;
    PSFS_CK(launch_likelihood(la, PSFS_MAP_F32, true, h->stream));
    return PSFS_OK;
}

psfs_status psfs_get_log_ratio(psfs_handle *h, const uint8_t *images, void *map_out)
{
    if (!h) return fail(PSFS_ERR_INVALID_ARG, "handle is NULL");
    if (!images || !aligned(images, 16)) return fail(PSFS_ERR_INVALID_ARG, "images NULL or not 16-byte aligned");
    if (!map_out || !aligned(map_out, 16)) return fail(PSFS_ERR_INVALID_ARG, "map_out NULL or not 16-byte aligned");
    if (!h->bg_ready) return fail(PSFS_ERR_NOT_READY, "psfs_set_background has not succeeded");
    DeviceGuard guard(h->device);
    LikelihoodArgs la{};
    la.img = images;
    la.mean = h->bg_mean;
    la.hinv = h->bg_hinv;
    la.n_pix = h->n_pix;
    la.c0 = h->c0;
    la.sc = h->sc;
    la.out = map_out;   // the kernel psfs_reconstruct runs, into the caller's buffer
    la.zero_word = nullptr;
    la.status = h->d_words;
    PSFS_CK(launch_likelihood(la, h->params.map_dtype, false, h->stream));
    return PSFS_OK;
}

static void fill_backward_args(psfs_handle *h, BackwardArgs &b);

// The owner lists of the pixel pass, built on the handle's stream by the
// first adjoint call (they depend on the grid and the rig only).
static psfs_status ensure_owner_lists(psfs_handle *h)
{
    if (h->own_ready) return PSFS_OK;
    if (!owner_lists_supported(h->fuse, h->n_pix))
        return fail(PSFS_ERR_INVALID_ARG, "adjoint: n_voxels * n_cams must be below 2^32");
    const uint64_t n_vox = (uint64_t)h->grid.nx * h->grid.ny * h->grid.nz;
    const size_t n_chunks = (size_t)(h->n_pix + 1 + 4095) / 4096;
    if (!h->own_off) {
        if (cudaMalloc(&h->own_off, ((size_t)h->n_pix + 1) * sizeof(uint32_t)) != cudaSuccess ||
            cudaMalloc(&h->own_cnt, (size_t)h->n_pix * sizeof(uint32_t)) != cudaSuccess ||
            cudaMalloc(&h->own_sums, n_chunks * sizeof(uint32_t)) != cudaSuccess ||
            cudaMalloc(&h->own_vox, std::max<size_t>(1, n_vox * (size_t)h->n_cams) * sizeof(uint32_t)) !=
                cudaSuccess) {
            cudaGetLastError();
            return fail(PSFS_ERR_NOMEM, "adjoint owner lists");
        }
    }
    FuseArgs fa = h->fuse;
    PSFS_CK(launch_build_owners(fa, h->n_pix, h->own_cnt, h->own_sums, h->own_off, h->own_vox, h->stream));
    h->own_ready = true;
    return PSFS_OK;
}

static psfs_status enqueue_backward(psfs_handle *h, const uint8_t *images, const float *slm, const float *d_occ,
                                    float *d_slm, float *d_mean, float *d_var)
{
    const uint64_t n_vox = (uint64_t)h->grid.nx * h->grid.ny * h->grid.nz;
    if (!h->dl) {
        if (cudaMalloc(&h->dl, n_vox * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return fail(PSFS_ERR_NOMEM, "adjoint scratch");
        }
    }
    psfs_status st = ensure_owner_lists(h);
    if (st != PSFS_OK) return st;
    BackwardArgs b;
    fill_backward_args(h, b);
    b.d_occ = d_occ;
    b.dl = h->dl;
    b.img = images;
    b.slm = slm;
    b.d_slm = d_slm;
    b.d_mean = d_mean;
    b.d_var = d_var;
    // recompute the forward maps
    if (images) {
        LikelihoodArgs la{};
        la.img = images;
        la.mean = h->bg_mean;
        la.hinv = h->bg_hinv;
        la.n_pix = h->n_pix;
        la.c0 = h->c0;
        la.sc = h->sc;
        la.out = h->maps;
        la.zero_word = nullptr;
        la.status = h->d_words;
        ProfScope ps(h, PSFS_STAGE_LIKELIHOOD);
        PSFS_CK(launch_likelihood(la, h->params.map_dtype, false, h->stream));
    } else {
        SlmToMapArgs sa{};
        sa.slm = slm;
        sa.n_pix = h->n_pix;
        sa.da = b.da;
        sa.one_minus_pd = b.one_minus_pd;
        sa.db = b.db;
        sa.one_minus_q = b.one_minus_q;
        sa.out = h->maps;
        sa.zero_word = nullptr;
        ProfScope ps(h, PSFS_STAGE_LIKELIHOOD);
        PSFS_CK(launch_slm_to_map(sa, h->params.map_dtype, h->stream));
    }
    {
        ProfScope ps(h, PSFS_STAGE_BACKWARD_VOXEL);
        FuseShape direct = h->shape;
        direct.staged = 0;   // the voxel pass uses the tile plan of either kernel with direct gathers
        PSFS_CK(launch_backward_voxel(b, direct, h->params.map_dtype, h->stream));
    }
    {
        ProfScope ps(h, PSFS_STAGE_BACKWARD_PIXEL);
        PSFS_CK(launch_owner_pixel(b, h->own_off, h->own_vox, h->stream));
    }
    return PSFS_OK;
}

// The arguments of the adjoint that depend on the handle only.
static void fill_backward_args(psfs_handle *h, BackwardArgs &b)
{
    std::memset(&b, 0, sizeof(b));
    b.f = h->fuse;
    b.mean = h->bg_mean;
    b.hinv = h->bg_hinv;
    b.c0 = h->c0;
    b.sc = h->sc;
    const double pd = h->params.p_detect, q = 0.5 * (h->params.p_detect + h->params.p_false_alarm);
    b.da = (float)(2.0 * pd - 1.0);
    b.one_minus_pd = (float)(1.0 - pd);
    b.db = (float)(2.0 * q - 1.0);
    b.one_minus_q = (float)(1.0 - q);
    b.n_pix = h->n_pix;
    b.dl_stride = 1;
}

// Tile shape of the batched adjoint's voxel pass (a frame-group shape: lanes_x
// 8, voxels_z 4), planned once per handle on first use.
constexpr FuseShape kBwShape = {8, 4, 4, 0};

// The two dLoss/dL record buffers of the batched adjoint (group g in buffer
// g & 1) and the sequence streams it pipelines on.
// Frames per owner pass of the batched adjoint: two planes of kBwRecord-frame
// records, so that the owner lists, the background and d_mean / d_var are
// read once per 16 frames.
constexpr int kBwGroup = 2 * kBwRecord;

static psfs_status ensure_dl_records(psfs_handle *h)
{
    const uint64_t n_vox = (uint64_t)h->grid.nx * h->grid.ny * h->grid.nz;
    for (float **buf : {&h->dl_rec, &h->dl_rec2}) {
        if (*buf) continue;
        if (cudaMalloc(buf, (size_t)kBwGroup * n_vox * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return fail(PSFS_ERR_NOMEM, "adjoint sequence scratch");
        }
    }
    return seq_setup(h);
}

static psfs_status ensure_backward_group(psfs_handle *h)
{
    psfs_status st = ensure_dl_records(h);
    if (st != PSFS_OK) return st;
    if (!h->bw_maps) {
        if (cudaMalloc(&h->bw_maps, (size_t)h->n_pix * kBwRecord * h->map_elem) != cudaSuccess) {
            cudaGetLastError();
            return fail(PSFS_ERR_NOMEM, "adjoint sequence maps");
        }
    }
    if (!h->bw_tiles) {
        std::vector<uint64_t> tiles;
        std::vector<int4> tilecam;
        FuseArgs fa;
        plan_fuse(h->grid, h->cams.data(), h->n_cams, h->params, kBwShape, &fa, &tiles, &tilecam);
        if (cudaMalloc(&h->bw_tiles, std::max<size_t>(1, tiles.size()) * sizeof(uint64_t)) != cudaSuccess ||
            cudaMalloc(&h->bw_tilecam, std::max<size_t>(1, tilecam.size()) * sizeof(int4)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(h->bw_tiles);
            h->bw_tiles = nullptr;
            return fail(PSFS_ERR_NOMEM, "adjoint sequence tile plan");
        }
        PSFS_CK(cudaMemcpyAsync(h->bw_tiles, tiles.data(), tiles.size() * sizeof(uint64_t), cudaMemcpyHostToDevice,
                                h->stream));
        PSFS_CK(cudaMemcpyAsync(h->bw_tilecam, tilecam.data(), tilecam.size() * sizeof(int4),
                                cudaMemcpyHostToDevice, h->stream));
        PSFS_CK(cudaStreamSynchronize(h->stream));   // the host vectors go out of scope
        fa.tiles = h->bw_tiles;
        fa.tilecam = h->bw_tilecam;
        fa.maps = h->bw_maps;
        fa.tmap_ok = 0;
        fa.status = h->d_words;
        h->bw_fuse = fa;
    }
    return PSFS_OK;
}

// Frames in groups of kBwGroup = 16: frames 0-7 of a group fill the first
// plane of 8-frame records, frames 8-15 the second.  A plane of nf frames runs
// in units of 8, 4, 2 and 1 frames (the binary digits of nf, largest first,
// so that a unit of P frames starts at a record slot that is a multiple of
// P): per unit one likelihood pass over the background for its P frames
// (maps as one plane of P-frame records) and one voxel pass that gathers each
// map record once per (voxel, camera) and writes dLoss/dL of the P frames
// into their slots; then one pixel pass for the group's 16 frames.  The
// record buffers alternate between groups,
// so a group's likelihood and voxel passes (stream 0) overlap the previous
// group's pixel pass (stream 1).  Per frame the arithmetic is that of
// psfs_backward, so d_slm is bit-identical to it.
static psfs_status enqueue_backward_sequence(psfs_handle *h, int32_t n_frames, const uint8_t *images,
                                             const float *d_occ, float *d_slm, float *d_mean, float *d_var)
{
    const uint64_t n_vox = (uint64_t)h->grid.nx * h->grid.ny * h->grid.nz;
    psfs_status st = ensure_owner_lists(h);
    if (st == PSFS_OK) st = ensure_backward_group(h);
    if (st != PSFS_OK) return st;
    BackwardArgs b;
    fill_backward_args(h, b);
    b.d_mean = d_mean;
    b.d_var = d_var;
    const size_t frame_bytes = (size_t)h->n_pix * 3;
    // group g's records are formed on stream 0 (likelihood and voxel passes)
    // into buffer g & 1 while stream 1 runs group g - 1's pixel pass from the
    // other buffer; the pixel passes stay in group order on stream 1 (they
    // accumulate d_mean and d_var)
    cudaStream_t sa = h->seq_stream[0], sb = h->seq_stream[1];
    float *bufs[2] = {h->dl_rec, h->dl_rec2};
    PSFS_CK(cudaEventRecord(h->seq_ev_in, h->stream));
    PSFS_CK(cudaStreamWaitEvent(sa, h->seq_ev_in, 0));
    PSFS_CK(cudaStreamWaitEvent(sb, h->seq_ev_in, 0));
    for (int g = 0, g0 = 0; g0 < n_frames; ++g, g0 += kBwGroup) {
        const int nf = std::min(kBwGroup, n_frames - g0);
        const int q = g & 1;
        if (g >= 2) PSFS_CK(cudaStreamWaitEvent(sa, h->seq_ev_fused[q], 0));   // group g - 2's pixel pass is done with it
        for (int r = 0; r * kBwRecord < nf; ++r) {
            const int nr = std::min(kBwRecord, nf - r * kBwRecord);   // frames of record plane r
            for (int slot = 0, P = kBwRecord; P >= 1; P /= 2) {
                if (!(nr & P)) continue;
                const size_t f0 = (size_t)g0 + r * kBwRecord + slot;   // the unit's first frame
                LikelihoodArgs la{};
                la.img = images + f0 * frame_bytes;
                la.mean = h->bg_mean;
                la.hinv = h->bg_hinv;
                la.n_pix = h->n_pix;
                la.c0 = h->c0;
                la.sc = h->sc;
                la.out = h->bw_maps;
                la.zero_word = nullptr;
                la.status = h->d_words;
                la.img_fstride = (int64_t)frame_bytes;
                {
                    ProfScope ps(h, PSFS_STAGE_LIKELIHOOD, sa);
                    if (P > 1)
                        PSFS_CK(launch_likelihood_group(la, P, h->params.map_dtype, sa, 4));
                    else
                        PSFS_CK(launch_likelihood(la, h->params.map_dtype, false, sa));
                }
                BackwardArgs bv = b;
                bv.f = h->bw_fuse;
                bv.d_occ = d_occ + f0 * n_vox;
                bv.dl = bufs[q] + (size_t)r * kBwRecord * n_vox + slot;
                bv.dl_stride = kBwRecord;
                {
                    ProfScope ps(h, PSFS_STAGE_BACKWARD_VOXEL, sa);
                    if (P > 1)
                        PSFS_CK(launch_backward_voxel_group(bv, kBwShape, P, h->params.map_dtype, (int64_t)n_vox, sa));
                    else
                        PSFS_CK(launch_backward_voxel(bv, kBwShape, h->params.map_dtype, sa));
                }
                slot += P;
            }
        }
        PSFS_CK(cudaEventRecord(h->seq_ev_map[q], sa));
        PSFS_CK(cudaStreamWaitEvent(sb, h->seq_ev_map[q], 0));
        BackwardArgs bp = b;
        bp.dl = bufs[q];
        bp.dl_stride = kBwRecord;
        bp.img = images + (size_t)g0 * frame_bytes;
        bp.d_slm = d_slm ? d_slm + (size_t)g0 * h->n_pix : nullptr;
        {
            ProfScope ps(h, PSFS_STAGE_BACKWARD_PIXEL, sb);
            PSFS_CK(launch_owner_pixel_group(bp, h->own_off, h->own_vox, nf, (int64_t)frame_bytes, g0 > 0, sb));
        }
        PSFS_CK(cudaEventRecord(h->seq_ev_fused[q], sb));
    }
    PSFS_CK(cudaEventRecord(h->seq_ev_done[0], sa));
    PSFS_CK(cudaEventRecord(h->seq_ev_done[1], sb));
    PSFS_CK(cudaStreamWaitEvent(h->stream, h->seq_ev_done[0], 0));
    PSFS_CK(cudaStreamWaitEvent(h->stream, h->seq_ev_done[1], 0));
    return PSFS_OK;
}

psfs_status psfs_backward(psfs_handle *h, const uint8_t *images, const float *d_occ, float *d_slm,
                          float *d_mean, float *d_var)
{
    if (!h) return fail(PSFS_ERR_INVALID_ARG, "handle is NULL");
    if (!images || !aligned(images, 16)) return fail(PSFS_ERR_INVALID_ARG, "images NULL or not 16-byte aligned");
    if (!d_occ || !aligned(d_occ, 16)) return fail(PSFS_ERR_INVALID_ARG, "d_occ NULL or not 16-byte aligned");
    if ((d_slm && !aligned(d_slm, 16)) || (d_mean && !aligned(d_mean, 16)) || (d_var && !aligned(d_var, 16)))
        return fail(PSFS_ERR_INVALID_ARG, "gradient buffer not 16-byte aligned");
    if (!h->bg_ready) return fail(PSFS_ERR_NOT_READY, "psfs_set_background has not succeeded");
    DeviceGuard guard(h->device);
    return enqueue_backward(h, images, nullptr, d_occ, d_slm, d_mean, d_var);
}

psfs_status psfs_backward_sequence(psfs_handle *h, int32_t n_frames, const uint8_t *images, const float *d_occ,
                                   float *d_slm, float *d_mean, float *d_var)
{
    if (!h) return fail(PSFS_ERR_INVALID_ARG, "handle is NULL");
    if (n_frames < 0) return fail(PSFS_ERR_INVALID_ARG, "n_frames < 0");
    if (n_frames == 0) return PSFS_OK;
    if (!images || !aligned(images, 16)) return fail(PSFS_ERR_INVALID_ARG, "images NULL or not 16-byte aligned");
    if ((h->n_pix * 3) % 16 != 0) return fail(PSFS_ERR_INVALID_ARG, "frame size not a multiple of 16 bytes");
    const uint64_t n_vox = (uint64_t)h->grid.nx * h->grid.ny * h->grid.nz;
    if (n_vox % 4 != 0) return fail(PSFS_ERR_INVALID_ARG, "voxel count not a multiple of 4");
    if (!d_occ || !aligned(d_occ, 16)) return fail(PSFS_ERR_INVALID_ARG, "d_occ NULL or not 16-byte aligned");
    if ((d_slm && !aligned(d_slm, 16)) || (d_mean && !aligned(d_mean, 16)) || (d_var && !aligned(d_var, 16)))
        return fail(PSFS_ERR_INVALID_ARG, "gradient buffer not 16-byte aligned");
    if (!h->bg_ready) return fail(PSFS_ERR_NOT_READY, "psfs_set_background has not succeeded");
    DeviceGuard guard(h->device);
    return enqueue_backward_sequence(h, n_frames, images, d_occ, d_slm, d_mean, d_var);
}

// The adjoint from the forward's own occupancy: dLoss/dL = d_occ occ (1 - occ)
// elementwise (no recomputed maps, no voxel pass), then the pixel passes of
// psfs_backward (one frame) or psfs_backward_sequence (groups of 16 frames in
// two planes of 8-frame records).
static psfs_status enqueue_backward_from_occupancy(psfs_handle *h, int32_t n_frames, const uint8_t *images,
                                                   const float *occupancy, const float *d_occ, float *d_slm,
                                                   float *d_mean, float *d_var)
{
    const uint64_t n_vox = (uint64_t)h->grid.nx * h->grid.ny * h->grid.nz;
    psfs_status st = ensure_owner_lists(h);
    if (st != PSFS_OK) return st;
    if (n_frames == 1 && !h->dl) {
        if (cudaMalloc(&h->dl, n_vox * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return fail(PSFS_ERR_NOMEM, "adjoint scratch");
        }
    }
    BackwardArgs b;
    fill_backward_args(h, b);
    b.d_mean = d_mean;
    b.d_var = d_var;
    if (n_frames == 1) {
        b.dl = h->dl;
        b.img = images;
        b.d_slm = d_slm;
        {
            ProfScope ps(h, PSFS_STAGE_BACKWARD_VOXEL);
            PSFS_CK(launch_dl_from_occ(occupancy, d_occ, h->dl, (int64_t)n_vox, 1, 1, h->stream));
        }
        ProfScope ps(h, PSFS_STAGE_BACKWARD_PIXEL);
        PSFS_CK(launch_owner_pixel(b, h->own_off, h->own_vox, h->stream));
        return PSFS_OK;
    }
    // group g's records (stream 0) into buffer g & 1 while stream 1 runs
    // group g - 1's pixel pass from the other buffer
    st = ensure_dl_records(h);
    if (st != PSFS_OK) return st;
    const size_t frame_bytes = (size_t)h->n_pix * 3;
    cudaStream_t sa = h->seq_stream[0], sb = h->seq_stream[1];
    float *bufs[2] = {h->dl_rec, h->dl_rec2};
    PSFS_CK(cudaEventRecord(h->seq_ev_in, h->stream));
    PSFS_CK(cudaStreamWaitEvent(sa, h->seq_ev_in, 0));
    PSFS_CK(cudaStreamWaitEvent(sb, h->seq_ev_in, 0));
    for (int g = 0, g0 = 0; g0 < n_frames; ++g, g0 += kBwGroup) {
        const int nf = std::min(kBwGroup, n_frames - g0);
        const int q = g & 1;
        if (g >= 2) PSFS_CK(cudaStreamWaitEvent(sa, h->seq_ev_fused[q], 0));
        for (int r = 0; r * kBwRecord < nf; ++r) {
            const size_t f0 = (size_t)g0 + r * kBwRecord;
            ProfScope ps(h, PSFS_STAGE_BACKWARD_VOXEL, sa);
            PSFS_CK(launch_dl_from_occ(occupancy + f0 * n_vox, d_occ + f0 * n_vox,
                                       bufs[q] + (size_t)r * kBwRecord * n_vox, (int64_t)n_vox,
                                       std::min(kBwRecord, nf - r * kBwRecord), kBwRecord, sa));
        }
        PSFS_CK(cudaEventRecord(h->seq_ev_map[q], sa));
        PSFS_CK(cudaStreamWaitEvent(sb, h->seq_ev_map[q], 0));
        BackwardArgs bp = b;
        bp.dl = bufs[q];
        bp.dl_stride = kBwRecord;
        bp.img = images + (size_t)g0 * frame_bytes;
        bp.d_slm = d_slm ? d_slm + (size_t)g0 * h->n_pix : nullptr;
        {
            ProfScope ps(h, PSFS_STAGE_BACKWARD_PIXEL, sb);
            PSFS_CK(launch_owner_pixel_group(bp, h->own_off, h->own_vox, nf, (int64_t)frame_bytes, g0 > 0, sb));
        }
        PSFS_CK(cudaEventRecord(h->seq_ev_fused[q], sb));
    }
    PSFS_CK(cudaEventRecord(h->seq_ev_done[0], sa));
    PSFS_CK(cudaEventRecord(h->seq_ev_done[1], sb));
    PSFS_CK(cudaStreamWaitEvent(h->stream, h->seq_ev_done[0], 0));
    PSFS_CK(cudaStreamWaitEvent(h->stream, h->seq_ev_done[1], 0));
    return PSFS_OK;
}

psfs_status psfs_backward_from_occupancy(psfs_handle *h, int32_t n_frames, const uint8_t *images,
                                         const float *occupancy, const float *d_occ, float *d_slm, float *d_mean,
                                         float *d_var)
{
    if (!h) return fail(PSFS_ERR_INVALID_ARG, "handle is NULL");
    if (n_frames < 0) return fail(PSFS_ERR_INVALID_ARG, "n_frames < 0");
    if (n_frames == 0) return PSFS_OK;
    if (!images || !aligned(images, 16)) return fail(PSFS_ERR_INVALID_ARG, "images NULL or not 16-byte aligned");
    if (n_frames > 1 && (h->n_pix * 3) % 16 != 0)
        return fail(PSFS_ERR_INVALID_ARG, "frame size not a multiple of 16 bytes");
    const uint64_t n_vox = (uint64_t)h->grid.nx * h->grid.ny * h->grid.nz;
    if (n_frames > 1 && n_vox % 4 != 0) return fail(PSFS_ERR_INVALID_ARG, "voxel count not a multiple of 4");
    if (!occupancy || !aligned(occupancy, 16))
        return fail(PSFS_ERR_INVALID_ARG, "occupancy NULL or not 16-byte aligned");
    if (!d_occ || !aligned(d_occ, 16)) return fail(PSFS_ERR_INVALID_ARG, "d_occ NULL or not 16-byte aligned");
    if ((d_slm && !aligned(d_slm, 16)) || (d_mean && !aligned(d_mean, 16)) || (d_var && !aligned(d_var, 16)))
        return fail(PSFS_ERR_INVALID_ARG, "gradient buffer not 16-byte aligned");
    if (!h->bg_ready) return fail(PSFS_ERR_NOT_READY, "psfs_set_background has not succeeded");
    DeviceGuard guard(h->device);
    return enqueue_backward_from_occupancy(h, n_frames, images, occupancy, d_occ, d_slm, d_mean, d_var);
}

psfs_status psfs_backward_slm(psfs_handle *h, const float *slm, const float *d_occ, float *d_slm)
{
    if (!h) return fail(PSFS_ERR_INVALID_ARG, "handle is NULL");
    if (!slm || !aligned(slm, 16)) return fail(PSFS_ERR_INVALID_ARG, "slm NULL or not 16-byte aligned");
    if (!d_occ || !aligned(d_occ, 16)) return fail(PSFS_ERR_INVALID_ARG, "d_occ NULL or not 16-byte aligned");
    if (!d_slm || !aligned(d_slm, 16)) return fail(PSFS_ERR_INVALID_ARG, "d_slm NULL or not 16-byte aligned");
    DeviceGuard guard(h->device);
    return enqueue_backward(h, nullptr, slm, d_occ, d_slm, nullptr, nullptr);
}

psfs_status psfs_set_fuse_config(psfs_handle *h, const psfs_fuse_config *cfg)
{
    if (!h || !cfg) return fail(PSFS_ERR_INVALID_ARG, "NULL argument");
    const FuseShape shape = {cfg->lanes_x, cfg->warps, cfg->voxels_z, cfg->staged};
    if (!fuse_shape_supported(shape)) return fail(PSFS_ERR_INVALID_ARG, "unsupported fuse tile shape");
    if (cfg->seq_likelihood_ctas < 0 || cfg->seq_likelihood_ctas > 4)
        return fail(PSFS_ERR_INVALID_ARG, "seq_likelihood_ctas outside [0, 4]");
    const bool own = cfg->seq_lanes_x > 0 || cfg->seq_voxels_z > 0;
    const FuseShape sshape = own ? FuseShape{cfg->seq_lanes_x, 4, cfg->seq_voxels_z, 0} : shape;
    if (own && !fuse_shape_supported(sshape))
        return fail(PSFS_ERR_INVALID_ARG, "unsupported sequence tile shape (seq_lanes_x, seq_voxels_z)");
    if (cfg->seq_record_bytes != 0 && cfg->seq_record_bytes != 32 && cfg->seq_record_bytes != 64)
        return fail(PSFS_ERR_INVALID_ARG, "seq_record_bytes: 0, 32 or 64");
    const int rec = cfg->seq_record_bytes ? cfg->seq_record_bytes : h->seq_rec;
    if (cfg->frames_per_group < 0 ||
        (cfg->frames_per_group > 1 && !group_shape_supported(sshape, cfg->frames_per_group, (int)h->map_elem, rec)))
        return fail(PSFS_ERR_INVALID_ARG,
                    "frames_per_group: 0, 1, or 2 / 4 / 8 / 16 / 32 with staged 0, lanes_x 8 or 16, voxels_z 2 or 4 "
                    "(8 when a pixel record holds at most 8 frames per lane, 16 when at most 4)");
    DeviceGuard guard(h->device);
    PSFS_CK(cudaStreamSynchronize(h->stream));
    if (h->seq_stream[0]) {
        PSFS_CK(cudaStreamSynchronize(h->seq_stream[0]));
        PSFS_CK(cudaStreamSynchronize(h->seq_stream[1]));
    }
    if (cfg->seq_likelihood_ctas > 0) h->seq_lk_ctas = cfg->seq_likelihood_ctas;
    if (cfg->frames_per_group > 0) h->seq_group = cfg->frames_per_group;
    h->seq_rec = rec;
    psfs_status st = replan(h, shape);
    if (st != PSFS_OK) return st;
    if (own) return replan_seq(h, sshape);
    h->seq_own = false;
    return PSFS_OK;
}

psfs_status psfs_get_fuse_config(psfs_handle *h, psfs_fuse_config *cfg)
{
    if (!h || !cfg) return fail(PSFS_ERR_INVALID_ARG, "NULL argument");
    cfg->lanes_x = h->shape.lx;
    cfg->warps = h->shape.wy;
    cfg->voxels_z = h->shape.tz;
    cfg->staged = h->shape.staged;
    cfg->seq_likelihood_ctas = h->seq_lk_ctas;
    cfg->frames_per_group = h->seq_group;
    cfg->cameras_per_block = 1;
    cfg->seq_lanes_x = seq_shape_of(h).lx;
    cfg->seq_voxels_z = seq_shape_of(h).tz;
    cfg->seq_record_bytes = h->seq_rec;
    return PSFS_OK;
}

psfs_status psfs_autotune(psfs_handle *h, const uint8_t *images, int32_t reps, psfs_fuse_config *best,
                          float *candidate_ms)
{
    if (!h) return fail(PSFS_ERR_INVALID_ARG, "handle is NULL");
    if (!images || !aligned(images, 16)) return fail(PSFS_ERR_INVALID_ARG, "images NULL or not 16-byte aligned");
    if (reps < 1) return fail(PSFS_ERR_INVALID_ARG, "reps < 1");
    if (!h->bg_ready) return fail(PSFS_ERR_NOT_READY, "psfs_set_background has not succeeded");
    DeviceGuard guard(h->device);
    const uint64_t n_vox = (uint64_t)h->grid.nx * h->grid.ny * h->grid.nz;
    // scratch: occupancy of kTuneFrames frames, kTuneFrames lists of
    // n_vox / kTuneFrames entries (the sequence timings; a frame with more
    // occupied voxels only sets the capacity bit, cleared below) and the
    // counts; two groups of 32 frames for grids up to 2^23 voxels, one above
    const int kTuneFrames = n_vox <= (1ull << 23) ? 2 * kMaxGroup : kMaxGroup;
    const uint32_t seq_cap = (uint32_t)std::max<uint64_t>(1, n_vox / kTuneFrames);
    float *occ = nullptr;
    uint32_t *list = nullptr, *tcounts = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&occ, kTuneFrames * n_vox * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&list, n_vox * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&tcounts, kTuneFrames * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(occ);
        cudaFree(list);
        return fail(PSFS_ERR_NOMEM, "autotune scratch");
    }
    psfs_status st = PSFS_OK;
    FuseShape best_shape = h->shape;
    float best_ms = 1e30f;
    // the candidates, in the order of candidate_ms: direct tiles (lanes_x 8,
    // 16, 32; voxels_z 2, 4, 8, 16), then staged ones (voxels_z 8, 16)
    FuseShape cands[PSFS_N_FUSE_CANDIDATES];
    {
        int n = 0;
        for (int lx : {8, 16, 32})
            for (int tz : {2, 4, 8, 16}) cands[n++] = FuseShape{lx, 4, tz, 0};
        for (int lx : {8, 16, 32})
            for (int tz : {8, 16}) cands[n++] = FuseShape{lx, 4, tz, 1};
    }
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = fail(PSFS_ERR_CUDA, "cudaEventCreate");
    // the maps of this frame, once: only the fuse kernel depends on the shape
    if (st == PSFS_OK) st = enqueue_reconstruct(h, images, occ, list, (uint32_t)n_vox, h->d_words + 3);
    for (int cand = 0; cand < PSFS_N_FUSE_CANDIDATES && st == PSFS_OK; ++cand) {
            const FuseShape shape = cands[cand];
            if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
                st = fail(PSFS_ERR_CUDA, "autotune sync");
                break;
            }
            st = replan(h, shape);
            if (st != PSFS_OK) break;
            FuseArgs fa;
            fill_fuse_args(h, occ, list, (uint32_t)n_vox, h->d_words + 3, &fa);
            cudaError_t err = launch_fuse(fa, shape, h->params.map_dtype, h->stream);   // warm-up
            if (err == cudaSuccess) err = cudaEventRecord(e0, h->stream);
            for (int r = 0; r < reps && err == cudaSuccess; ++r) {
                err = cudaMemsetAsync(h->d_words + 3, 0, sizeof(uint32_t), h->stream);
                if (err == cudaSuccess) err = launch_fuse(fa, shape, h->params.map_dtype, h->stream);
            }
            if (err == cudaSuccess) err = cudaEventRecord(e1, h->stream);
            if (err == cudaSuccess) err = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
            if (err != cudaSuccess) {
                st = fail_cuda(err, "autotune timing");
                break;
            }
            if (candidate_ms) candidate_ms[cand] = ms / (float)reps;
            if (ms < best_ms) {
                best_ms = ms;
                best_shape = shape;
            }
    }
    // second stage: the sequence path, timed on kTuneFrames frames (distinct
    // outputs; copies of the one frame at distinct addresses, so that the
    // images come from HBM as in a real sequence, or the same buffer when
    // there is no room for the copies) per repetition: CTAs per SM of the
    // likelihood grid (1 to 4) with one frame per launch, then frame groups of
    // 2, 4, 8, 16 and 32 frames with the direct tile shapes that support them
    const size_t frame_bytes = (size_t)h->n_pix * 3;
    uint8_t *tune_imgs = nullptr;
    size_t tune_stride = 0;
    if (st == PSFS_OK && frame_bytes % 16 == 0) {   // frame strides of bulk copies: 16-byte multiples
        if (cudaMalloc(&tune_imgs, (size_t)kTuneFrames * frame_bytes) == cudaSuccess) {
            for (int f = 0; f < kTuneFrames && st == PSFS_OK; ++f)
                if (cudaMemcpyAsync(tune_imgs + (size_t)f * frame_bytes, images, frame_bytes,
                                    cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
                    st = fail(PSFS_ERR_CUDA, "autotune frame copies");
            tune_stride = frame_bytes;
        } else {
            cudaGetLastError();
            tune_imgs = nullptr;
        }
    }
    const uint8_t *seq_imgs = tune_imgs ? tune_imgs : images;
    auto time_sequence = [&](int lk, int group, float *ms_out) -> psfs_status {
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(PSFS_ERR_CUDA, "autotune sync");
        psfs_status s2 = enqueue_sequence(h, kTuneFrames, seq_imgs, tune_stride, occ, n_vox, list, seq_cap,
                                          seq_cap, tcounts, 1, lk, group);   // warm-up (allocates group buffers)
        if (s2 != PSFS_OK) return s2;
        cudaError_t err = cudaEventRecord(e0, h->stream);
        for (int r = 0; r < reps && s2 == PSFS_OK && err == cudaSuccess; ++r)
            s2 = enqueue_sequence(h, kTuneFrames, seq_imgs, tune_stride, occ, n_vox, list, seq_cap, seq_cap,
                                  tcounts, 1, lk, group);
        if (s2 != PSFS_OK) return s2;
        if (err == cudaSuccess) err = cudaEventRecord(e1, h->stream);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err != cudaSuccess) return fail_cuda(err, "autotune sequence timing");
        *ms_out = ms;
        return PSFS_OK;
    };
    if (st == PSFS_OK) st = replan(h, best_shape);   // the best shape for one frame per call
    h->seq_own = false;
    float best_seq = 1e30f;
    int best_group = 1;
    int best_rec = 32;
    FuseShape best_seq_shape = best_shape;
    h->seq_rec = 32;
    for (int lk = 1; lk <= 4 && st == PSFS_OK; ++lk) {
        float ms = 0.0f;
        st = time_sequence(lk, 1, &ms);
        if (st == PSFS_OK && ms < best_seq) {
            best_seq = ms;
            h->seq_lk_ctas = lk;
        }
    }
    const int group_lx = (best_shape.lx == 16) ? 16 : 8;
    const int groups[5] = {2, 4, 8, 16, kMaxGroup};
    for (int gi = 0; gi < 5 && st == PSFS_OK; ++gi) {
        for (int rec : {32, 64}) {
            // 64-byte records only differ once a group fills more than 32 bytes per pixel
            if (rec == 64 && groups[gi] * (int)h->map_elem <= 32) continue;
            for (int tz : {2, 4, 8, 16}) {
                if (st != PSFS_OK) break;
                const FuseShape gshape = {group_lx, 4, tz, 0};
                if (!group_shape_supported(gshape, groups[gi], (int)h->map_elem, rec)) continue;
                st = replan_seq(h, gshape);
                h->seq_rec = rec;
                for (int lk = 1; lk <= 3 && st == PSFS_OK; ++lk) {
                    float ms = 0.0f;
                    st = time_sequence(lk, groups[gi], &ms);
                    if (st == PSFS_OK && ms < best_seq) {
                        best_seq = ms;
                        best_group = groups[gi];
                        best_rec = rec;
                        best_seq_shape = gshape;
                        h->seq_lk_ctas = lk;
                    }
                }
            }
        }
    }
    h->seq_group = best_group;
    h->seq_rec = best_rec;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(h->stream);
    cudaFree(occ);
    cudaFree(list);
    cudaFree(tcounts);
    cudaFree(tune_imgs);
    cudaMemsetAsync(h->d_words, 0, sizeof(uint32_t), h->stream);   // the scratch list never overflows
    if (st != PSFS_OK) return st;
    // one frame per call keeps the best single-frame shape; the sequence path
    // gets its own plan when frame groups won with another shape
    h->seq_own = false;
    if (best_group > 1 && !(best_seq_shape.lx == best_shape.lx && best_seq_shape.tz == best_shape.tz &&
                            best_seq_shape.staged == best_shape.staged)) {
        st = replan_seq(h, best_seq_shape);
        if (st != PSFS_OK) return st;
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[tune_key(h)] = Tuned{best_shape, h->seq_lk_ctas, h->seq_group, h->seq_own, h->seq_shape, h->seq_rec};
    }
    if (best) psfs_get_fuse_config(h, best);
    return PSFS_OK;
}

psfs_status psfs_tune_cache_save(const char *path)
{
    if (!path) return fail(PSFS_ERR_INVALID_ARG, "path is NULL");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    FILE *fp = std::fopen(path, "w");
    if (!fp) return fail(PSFS_ERR_INVALID_ARG, "tune cache file cannot be opened for writing");
    bool ok = std::fprintf(fp, "psfs-tune 1\n") > 0;
    for (const auto &kv : g_tuned) {
        const TuneKey &k = kv.first;
        const Tuned &t = kv.second;
        ok = ok && std::fprintf(fp, "%d %d %d %d %d %d %d  %d %d %d %d  %d %d  %d %d %d %d %d  %d\n", std::get<0>(k),
                                std::get<1>(k), std::get<2>(k), std::get<3>(k), std::get<4>(k), std::get<5>(k),
                                std::get<6>(k), t.shape.lx, t.shape.wy, t.shape.tz, t.shape.staged, t.seq_lk_ctas,
                                t.seq_group, t.seq_own ? 1 : 0, t.seq_shape.lx, t.seq_shape.wy, t.seq_shape.tz,
                                t.seq_shape.staged, t.seq_rec) > 0;
    }
    ok = (std::fclose(fp) == 0) && ok;
    if (!ok) return fail(PSFS_ERR_INVALID_ARG, "tune cache file could not be written");
    return PSFS_OK;
}

psfs_status psfs_tune_cache_load(const char *path)
{
    if (!path) return fail(PSFS_ERR_INVALID_ARG, "path is NULL");
    FILE *fp = std::fopen(path, "r");
    if (!fp) return fail(PSFS_ERR_INVALID_ARG, "tune cache file cannot be opened for reading");
    std::map<TuneKey, Tuned> add;
    char line[512];
    int lineno = 0;
    bool ok = true;
    static thread_local char msg[128];
    auto bad = [&](const char *why) {
        std::snprintf(msg, sizeof(msg), "tune cache line %d: %s", lineno, why);
        ok = false;
    };
    while (ok && std::fgets(line, sizeof(line), fp)) {
        ++lineno;
        if (lineno == 1) {
            int version = 0;
            if (std::sscanf(line, "psfs-tune %d", &version) != 1 || version != 1) bad("not a psfs-tune 1 file");
            continue;
        }
        bool blank = true;
        for (const char *c = line; *c; ++c) blank = blank && (*c == ' ' || *c == '\t' || *c == '\n' || *c == '\r');
        if (blank) continue;
        int v[19], used = 0;
        if (std::sscanf(line, "%d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d%n", &v[0], &v[1], &v[2],
                        &v[3], &v[4], &v[5], &v[6], &v[7], &v[8], &v[9], &v[10], &v[11], &v[12], &v[13], &v[14],
                        &v[15], &v[16], &v[17], &v[18], &used) != 19) {
            bad("not 19 integers");
            break;
        }
        for (const char *c = line + used; *c; ++c)
            if (!(*c == ' ' || *c == '\t' || *c == '\n' || *c == '\r')) {
                bad("trailing characters");
                break;
            }
        if (!ok) break;
        const int nx = v[0], ny = v[1], nz = v[2], K = v[3], W = v[4], H = v[5], dt = v[6];
        if (nx < 1 || ny < 1 || nz < 1 || nx > (1 << 24) || ny > (1 << 24) || nz > (1 << 24) || K < 1 ||
            K > PSFS_MAX_CAMS || W < 1 || H < 1 || (dt != PSFS_MAP_F32 && dt != PSFS_MAP_F16 && dt != PSFS_MAP_BF16)) {
            bad("grid, camera count, image size or map type out of range");
            break;
        }
        Tuned t;
        t.shape = FuseShape{v[7], v[8], v[9], v[10]};
        t.seq_lk_ctas = v[11];
        t.seq_group = v[12];
        t.seq_own = v[13] != 0;
        t.seq_shape = FuseShape{v[14], v[15], v[16], v[17]};
        t.seq_rec = v[18];
        const int elem = dt == PSFS_MAP_F32 ? 4 : 2;
        const FuseShape &sshape = t.seq_own ? t.seq_shape : t.shape;
        if (!fuse_shape_supported(t.shape) || (v[13] != 0 && v[13] != 1) ||
            (t.seq_own && (!fuse_shape_supported(t.seq_shape) || t.seq_shape.staged != 0)) || t.seq_lk_ctas < 1 ||
            t.seq_lk_ctas > 4 || (t.seq_rec != 32 && t.seq_rec != 64) ||
            !(t.seq_group == 1 || group_shape_supported(sshape, t.seq_group, elem, t.seq_rec))) {
            bad("unsupported configuration");
            break;
        }
        if (!t.seq_own) t.seq_shape = t.shape;
        add[TuneKey(nx, ny, nz, K, W, H, dt)] = t;
    }
    if (ok && std::ferror(fp)) {
        std::snprintf(msg, sizeof(msg), "tune cache file could not be read");
        ok = false;
    }
    if (ok && lineno == 0) {
        std::snprintf(msg, sizeof(msg), "tune cache file is empty");
        ok = false;
    }
    std::fclose(fp);
    if (!ok) return fail(PSFS_ERR_INVALID_ARG, msg);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto &kv : add) g_tuned[kv.first] = kv.second;
    return PSFS_OK;
}

void psfs_tune_cache_clear(void)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned.clear();
}

int32_t psfs_tune_cache_entries(void)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return (int32_t)g_tuned.size();
}

psfs_status psfs_sync(psfs_handle *h)
{
    if (!h) return fail(PSFS_ERR_INVALID_ARG, "handle is NULL");
    DeviceGuard guard(h->device);
    PSFS_CK(cudaMemcpyAsync(h->h_words, h->d_words, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream));
    PSFS_CK(cudaMemsetAsync(h->d_words, 0, sizeof(uint32_t), h->stream));
    PSFS_CK(cudaStreamSynchronize(h->stream));
    const uint32_t w = h->h_words[0];
    if (w & kStatusBounds) return fail(PSFS_ERR_BOUNDS, "a bounds check failed; the access was skipped");
    if (w & kStatusCapacity) return fail(PSFS_ERR_CAPACITY, "voxel list capacity exceeded");
    if (w & kStatusTimeout) return fail(PSFS_ERR_TIMEOUT, "device wait timed out");
    return PSFS_OK;
}

psfs_status psfs_profile_enable(psfs_handle *h, int32_t max_launches)
{
    if (!h) return fail(PSFS_ERR_INVALID_ARG, "handle is NULL");
    if (max_launches < 0) return fail(PSFS_ERR_INVALID_ARG, "max_launches < 0");
    DeviceGuard guard(h->device);
    PSFS_CK(cudaStreamSynchronize(h->stream));
    prof_free(h);
    if (max_launches == 0) return PSFS_OK;
    h->prof_ev.resize(2 * (size_t)max_launches, nullptr);
    h->prof_stage.assign((size_t)max_launches, 0);
    for (auto &e : h->prof_ev) {
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) {
            prof_free(h);
            return fail_cuda(err, "cudaEventCreate");
        }
    }
    h->prof_cap = max_launches;
    return PSFS_OK;
}

psfs_status psfs_profile_read(psfs_handle *h, double *ms, int32_t *launches)
{
    if (!h || !ms || !launches) return fail(PSFS_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard guard(h->device);
    PSFS_CK(cudaStreamSynchronize(h->stream));
    for (int s = 0; s < PSFS_N_STAGES; ++s) {
        ms[s] = 0.0;
        launches[s] = 0;
    }
    for (int n = 0; n < h->prof_n; ++n) {
        float t = 0.0f;
        PSFS_CK(cudaEventElapsedTime(&t, h->prof_ev[2 * n], h->prof_ev[2 * n + 1]));
        ms[h->prof_stage[n]] += t;
        launches[h->prof_stage[n]] += 1;
    }
    h->prof_n = 0;
    return PSFS_OK;
}

void psfs_destroy(psfs_handle *h) { free_handle(h); }

}  // extern "C"

// ---------------------------------------------------------------------------
// batched persistent launch over many frames (form of the hot path with no
// counterpart in the paper, which runs one frame at a time)
// ---------------------------------------------------------------------------
struct psfs_batch {
    int device = 0;
    cudaStream_t user_stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    // the other streams of the frame-launch graph, and its fork and join events
    cudaStream_t cap_more[kBatchStreams - 1] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[kBatchStreams - 1] = {};
    int map_dtype = PSFS_MAP_F32;
    int launch = 0;               // 0: one persistent kernel; 1: a graph of per-frame launches
    std::vector<psfs_frame> frames;
    FuseShape shape = kDefaultFuseShape;
    BatchFrame *d_frames = nullptr;
    uint64_t *d_items = nullptr;
    int64_t n_items = 0;
    uint32_t *d_words = nullptr;   // [0] status, [16 ...] per-frame done counters
    uint32_t *h_words = nullptr;
    std::vector<void *> maps;
    std::vector<uint64_t *> tiles;
    std::vector<int4 *> tilecam;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int blocks = 0;
    uint64_t wait_ns = kWaitNs;   // limit of the fusion tiles' waits
    int hold_frame = -1;          // test hook: this frame's tiles wait for one chunk too many
    int cam_block = 1;            // cameras whose loads a fusion item issues together
};

namespace {

void batch_free_plan(psfs_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    for (auto p : b->tiles) cudaFree(p);
    for (auto p : b->tilecam) cudaFree(p);
    b->tiles.clear();
    b->tilecam.clear();
    cudaFree(b->d_frames);
    cudaFree(b->d_items);
    b->d_frames = nullptr;
    b->d_items = nullptr;
}

void batch_free(psfs_batch *b)
{
    if (!b) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    if (b->cap_stream) cudaStreamSynchronize(b->cap_stream);
    cudaStreamSynchronize(b->user_stream);
    batch_free_plan(b);
    for (auto p : b->maps) cudaFree(p);
    cudaFree(b->d_words);
    cudaFreeHost(b->h_words);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (int k = 0; k < kBatchStreams - 1; ++k) {
        if (b->cap_more[k]) cudaStreamDestroy(b->cap_more[k]);
        if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    cudaSetDevice(prev);
    delete b;
}

// Plans every frame for `shape`, builds the interleaved work list, uploads the
// descriptors and captures [zero the counters, batched kernel] in a graph.
psfs_status batch_build(psfs_batch *b, const FuseShape &shape)
{
    batch_free_plan(b);
    const int F = (int)b->frames.size();
    std::vector<BatchFrame> hf(F);
    std::vector<uint32_t> n_chunks(F), n_tiles(F);
    for (int f = 0; f < F; ++f) {
        const psfs_frame &fr = b->frames[f];
        psfs_handle *h = fr.handle;
        std::vector<uint64_t> tiles;
        std::vector<int4> tilecam;
        FuseArgs fa;
        plan_fuse(h->grid, h->cams.data(), h->n_cams, h->params, shape, &fa, &tiles, &tilecam);
        uint64_t *dt = nullptr;
        int4 *dtc = nullptr;
        if (cudaMalloc(&dt, tiles.size() * sizeof(uint64_t)) != cudaSuccess ||
            cudaMalloc(&dtc, tilecam.size() * sizeof(int4)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(dt);
            return fail(PSFS_ERR_NOMEM, "batch plan allocation");
        }
        b->tiles.push_back(dt);
        b->tilecam.push_back(dtc);
        PSFS_CK(cudaMemcpy(dt, tiles.data(), tiles.size() * sizeof(uint64_t), cudaMemcpyHostToDevice));
        PSFS_CK(cudaMemcpy(dtc, tilecam.data(), tilecam.size() * sizeof(int4), cudaMemcpyHostToDevice));
        fa.maps = b->maps[f];
        fa.tmap_ok = 0;   // batched items gather from global memory
        fa.tiles = dt;
        fa.tilecam = dtc;
        fa.occ = fr.occupancy;
        fa.list = fr.voxel_list;
        fa.capacity = fr.capacity;
        fa.count = fr.count;
        fa.status = b->d_words;
        BatchFrame &bf = hf[f];
        std::memset(&bf, 0, sizeof(bf));
        bf.fa = fa;
        bf.img = fr.images;
        bf.mean = h->bg_mean;
        bf.hinv = h->bg_hinv;
        bf.n_pix = h->n_pix;
        bf.n_chunks = (uint32_t)((h->n_pix + kBatchChunk - 1) / kBatchChunk);
        bf.wait_chunks = bf.n_chunks + (f == b->hold_frame ? 1u : 0u);
        bf.c0 = h->c0;
        bf.sc = h->sc;
        n_chunks[f] = bf.n_chunks;
        n_tiles[f] = (uint32_t)fa.n_tiles;
    }
    // work list: chunks of frame f interleaved with tiles of frame f - 1
    std::vector<uint64_t> items;
    for (int f = 0; f <= F; ++f) {
        const uint64_t nc = f < F ? n_chunks[f] : 0, nt = f > 0 ? n_tiles[f - 1] : 0;
        uint64_t ci = 0, ti = 0;
        while (ci < nc || ti < nt) {
            // take a chunk while chunks are ahead of tiles in proportion
            const bool take_chunk = ti >= nt || (ci < nc && ci * nt <= ti * nc);
            if (take_chunk) items.push_back(pack_item((uint32_t)f, 0, ci++));
            else items.push_back(pack_item((uint32_t)(f - 1), 1, ti++));
        }
    }
    b->n_items = (int64_t)items.size();
    if (cudaMalloc(&b->d_frames, hf.size() * sizeof(BatchFrame)) != cudaSuccess ||
        cudaMalloc(&b->d_items, std::max<size_t>(1, items.size()) * sizeof(uint64_t)) != cudaSuccess) {
        cudaGetLastError();
        return fail(PSFS_ERR_NOMEM, "batch descriptor allocation");
    }
    PSFS_CK(cudaMemcpy(b->d_frames, hf.data(), hf.size() * sizeof(BatchFrame), cudaMemcpyHostToDevice));
    if (!items.empty())
        PSFS_CK(cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(uint64_t), cudaMemcpyHostToDevice));
    BatchLaunch bl;
    bl.frames = b->d_frames;
    bl.items = b->d_items;
    bl.n_items = b->n_items;
    bl.done = b->d_words + 16;
    bl.status = b->d_words;
    bl.blocks = b->blocks;
    bl.wait_ns = b->wait_ns;
    PSFS_CK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemsetAsync(b->d_words + 16, 0, sizeof(uint32_t) * (size_t)F, b->cap_stream);
    if (e == cudaSuccess) e = launch_batch(bl, shape, b->cam_block, b->map_dtype, b->cap_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail_cuda(e, "batch capture");
    }
    if (e2 != cudaSuccess) return fail_cuda(e2, "cudaStreamEndCapture");
    b->graph = g;
    PSFS_CK(cudaGraphInstantiate(&b->exec, g, 0));
    b->shape = shape;
    b->launch = 0;
    return PSFS_OK;
}

// The other launch form: a graph of each frame's own likelihood and fusion
// launches (the kernels of psfs_reconstruct, each frame with its handle's
// one-frame tile shape, a direct one when that is staged, planned here so
// that later changes to the handles leave the graph valid), frame f on
// stream f mod kBatchStreams, so that frames' likelihoods run beside earlier
// frames' fusions and small frames share the GPU.  No device-side waits: the
// streams order each frame's two stages.
psfs_status batch_build_frames(psfs_batch *b)
{
    batch_free_plan(b);
    const int F = (int)b->frames.size();
    std::vector<FuseArgs> fas(F);
    std::vector<FuseShape> shapes(F);
    for (int f = 0; f < F; ++f) {
        const psfs_frame &fr = b->frames[f];
        psfs_handle *h = fr.handle;
        shapes[f] = h->shape.staged ? kDefaultFuseShape : h->shape;
        std::vector<uint64_t> tiles;
        std::vector<int4> tilecam;
        FuseArgs &fa = fas[f];
        plan_fuse(h->grid, h->cams.data(), h->n_cams, h->params, shapes[f], &fa, &tiles, &tilecam);
        uint64_t *dt = nullptr;
        int4 *dtc = nullptr;
        if (cudaMalloc(&dt, std::max<size_t>(1, tiles.size()) * sizeof(uint64_t)) != cudaSuccess ||
            cudaMalloc(&dtc, std::max<size_t>(1, tilecam.size()) * sizeof(int4)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(dt);
            return fail(PSFS_ERR_NOMEM, "batch plan allocation");
        }
        b->tiles.push_back(dt);
        b->tilecam.push_back(dtc);
        PSFS_CK(cudaMemcpy(dt, tiles.data(), tiles.size() * sizeof(uint64_t), cudaMemcpyHostToDevice));
        PSFS_CK(cudaMemcpy(dtc, tilecam.data(), tilecam.size() * sizeof(int4), cudaMemcpyHostToDevice));
        fa.maps = b->maps[f];
        fa.tmap_ok = 0;
        fa.tiles = dt;
        fa.tilecam = dtc;
        fa.occ = fr.occupancy;
        fa.list = fr.voxel_list;
        fa.capacity = fr.capacity;
        fa.count = fr.count;
        fa.status = b->d_words;
    }
    PSFS_CK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaEventRecord(b->ev_fork, b->cap_stream);
    for (int k = 0; k < kBatchStreams - 1 && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->cap_more[k], b->ev_fork, 0);
    for (int f = 0; f < F && e == cudaSuccess; ++f) {
        const psfs_frame &fr = b->frames[f];
        psfs_handle *h = fr.handle;
        const int k = f % kBatchStreams;
        cudaStream_t s = k == 0 ? b->cap_stream : b->cap_more[k - 1];
        LikelihoodArgs la{};
        la.img = fr.images;
        la.mean = h->bg_mean;
        la.hinv = h->bg_hinv;
        la.n_pix = h->n_pix;
        la.c0 = h->c0;
        la.sc = h->sc;
        la.out = b->maps[f];
        la.zero_word = fr.count;
        la.status = b->d_words;
        e = launch_likelihood(la, b->map_dtype, false, s);
        if (e == cudaSuccess) e = launch_fuse(fas[f], shapes[f], b->map_dtype, s);
    }
    for (int k = 0; k < kBatchStreams - 1 && e == cudaSuccess; ++k) {
        e = cudaEventRecord(b->ev_join[k], b->cap_more[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap_stream, b->ev_join[k], 0);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail_cuda(e, "batch frame-launch capture");
    }
    if (e2 != cudaSuccess) return fail_cuda(e2, "cudaStreamEndCapture");
    b->graph = g;
    PSFS_CK(cudaGraphInstantiate(&b->exec, g, 0));
    b->launch = 1;
    return PSFS_OK;
}

}  // namespace

extern "C" {

psfs_status psfs_batch_create(const psfs_frame *frames, int32_t n_frames, void *stream, psfs_batch **out)
{
    if (!out) return fail(PSFS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!frames || n_frames < 1 || n_frames > (1 << 23)) return fail(PSFS_ERR_INVALID_ARG, "frames / n_frames");
    const int dtype = frames[0].handle ? frames[0].handle->params.map_dtype : -1;
    for (int f = 0; f < n_frames; ++f) {
        const psfs_frame &fr = frames[f];
        if (!fr.handle) return fail(PSFS_ERR_INVALID_ARG, "frame without a handle");
        if (!fr.handle->bg_ready) return fail(PSFS_ERR_NOT_READY, "a frame's handle has no background");
        if (fr.handle->params.map_dtype != dtype) return fail(PSFS_ERR_INVALID_ARG, "frames differ in map_dtype");
        if (!fr.images || !aligned(fr.images, 16)) return fail(PSFS_ERR_INVALID_ARG, "frame images NULL or unaligned");
        psfs_status st = check_frame_outputs(fr.occupancy, fr.voxel_list, fr.capacity, fr.count);
        if (st != PSFS_OK) return st;
        if (fr.handle->device != frames[0].handle->device) return fail(PSFS_ERR_INVALID_ARG, "frames on different devices");
    }
    psfs_batch *b = new (std::nothrow) psfs_batch();
    if (!b) return fail(PSFS_ERR_NOMEM, "host allocation");
    b->device = frames[0].handle->device;
    b->user_stream = (cudaStream_t)stream;
    b->map_dtype = dtype;
    b->frames.assign(frames, frames + n_frames);
    DeviceGuard guard(b->device);
    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&b->d_words, sizeof(uint32_t) * (16 + (size_t)n_frames)) != cudaSuccess ||
        cudaMallocHost(&b->h_words, sizeof(uint32_t) * 16) != cudaSuccess) {
        cudaGetLastError();
        batch_free(b);
        return fail(PSFS_ERR_NOMEM, "batch allocation");
    }
    cudaMemset(b->d_words, 0, sizeof(uint32_t) * (16 + (size_t)n_frames));
    for (int k = 0; k < kBatchStreams - 1; ++k) {
        if (cudaStreamCreateWithFlags(&b->cap_more[k], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            batch_free(b);
            return fail(PSFS_ERR_CUDA, "batch streams");
        }
    }
    const size_t elem = dtype == PSFS_MAP_F32 ? 4 : 2;
    for (int f = 0; f < n_frames; ++f) {
        void *m = nullptr;
        if (cudaMalloc(&m, (size_t)frames[f].handle->n_pix * elem) != cudaSuccess) {
            cudaGetLastError();
            batch_free(b);
            return fail(PSFS_ERR_NOMEM, "batch map buffers");
        }
        b->maps.push_back(m);
    }
    psfs_status st = batch_build(b, frames[0].handle->shape.staged ? kDefaultFuseShape : frames[0].handle->shape);
    if (st != PSFS_OK) {
        batch_free(b);
        return st;
    }
    *out = b;
    return PSFS_OK;
}

psfs_status psfs_batch_run(psfs_batch *b)
{
    if (!b) return fail(PSFS_ERR_INVALID_ARG, "batch is NULL");
    DeviceGuard guard(b->device);
    PSFS_CK(cudaGraphLaunch(b->exec, b->user_stream));
    return PSFS_OK;
}

psfs_status psfs_batch_sync(psfs_batch *b)
{
    if (!b) return fail(PSFS_ERR_INVALID_ARG, "batch is NULL");
    DeviceGuard guard(b->device);
    PSFS_CK(cudaMemcpyAsync(b->h_words, b->d_words, sizeof(uint32_t), cudaMemcpyDeviceToHost, b->user_stream));
    PSFS_CK(cudaMemsetAsync(b->d_words, 0, sizeof(uint32_t), b->user_stream));
    PSFS_CK(cudaStreamSynchronize(b->user_stream));
    const uint32_t w = b->h_words[0];
    if (w & kStatusBounds) return fail(PSFS_ERR_BOUNDS, "a bounds check failed; the access was skipped");
    if (w & kStatusTimeout) return fail(PSFS_ERR_TIMEOUT, "a batched work item timed out waiting for its frame");
    if (w & kStatusCapacity) return fail(PSFS_ERR_CAPACITY, "voxel list capacity exceeded");
    return PSFS_OK;
}

psfs_status psfs_batch_set_config(psfs_batch *b, const psfs_fuse_config *cfg)
{
    if (!b || !cfg) return fail(PSFS_ERR_INVALID_ARG, "NULL argument");
    if (cfg->batch_launch != 0 && cfg->batch_launch != 1) return fail(PSFS_ERR_INVALID_ARG, "batch_launch: 0 or 1");
    if (cfg->batch_launch == 1) {
        DeviceGuard guard(b->device);
        PSFS_CK(cudaStreamSynchronize(b->user_stream));
        return batch_build_frames(b);
    }
    const FuseShape shape = {cfg->lanes_x, cfg->warps, cfg->voxels_z, 0};
    const int cb = cfg->cameras_per_block > 0 ? cfg->cameras_per_block : 1;
    if (cfg->staged != 0 || !batch_shape_supported(shape, cb))
        return fail(PSFS_ERR_INVALID_ARG,
                    "unsupported batch tile shape or camera block (staged is not available in a batch)");
    DeviceGuard guard(b->device);
    PSFS_CK(cudaStreamSynchronize(b->user_stream));
    const int old_cb = b->cam_block;
    b->cam_block = cb;
    const psfs_status st = batch_build(b, shape);
    if (st != PSFS_OK) b->cam_block = old_cb;
    return st;
}

psfs_status psfs_batch_autotune(psfs_batch *b, int32_t reps, psfs_fuse_config *best, float *candidate_ms)
{
    if (!b || reps < 1) return fail(PSFS_ERR_INVALID_ARG, "batch NULL or reps < 1");
    DeviceGuard guard(b->device);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PSFS_CK(cudaEventCreate(&e0));
    PSFS_CK(cudaEventCreate(&e1));
    // candidates (order of candidate_ms): lanes_x 8, 16, 32 x voxels_z 8, 16 with
    // one camera per load block, then camera blocks of 2 (lanes_x 8, 16 x
    // voxels_z 4, 8) and of 4 (lanes_x 8, 16, voxels_z 4)
    struct Cand {
        int lx, tz, cb;
    };
    const Cand cands[kBatchCandidates - 1] = {{8, 8, 1}, {8, 16, 1}, {16, 8, 1}, {16, 16, 1}, {32, 8, 1}, {32, 16, 1},
                                              {8, 4, 2}, {8, 8, 2},  {16, 4, 2}, {16, 8, 2},  {8, 4, 4},  {16, 4, 4}};
    FuseShape best_shape = b->shape;
    int best_cb = b->cam_block;
    float best_ms = 1e30f;
    psfs_status st = PSFS_OK;
    for (int cand = 0; cand < kBatchCandidates - 1 && st == PSFS_OK; ++cand) {
        const FuseShape shape = {cands[cand].lx, 4, cands[cand].tz, 0};
        if (cudaStreamSynchronize(b->user_stream) != cudaSuccess) {
            st = fail(PSFS_ERR_CUDA, "batch autotune sync");
            break;
        }
        b->cam_block = cands[cand].cb;
        st = batch_build(b, shape);
        if (st != PSFS_OK) break;
        cudaError_t err = cudaGraphLaunch(b->exec, b->user_stream);   // warm-up
        if (err == cudaSuccess) err = cudaEventRecord(e0, b->user_stream);
        for (int r = 0; r < reps && err == cudaSuccess; ++r) err = cudaGraphLaunch(b->exec, b->user_stream);
        if (err == cudaSuccess) err = cudaEventRecord(e1, b->user_stream);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err != cudaSuccess) {
            st = fail_cuda(err, "batch autotune timing");
            break;
        }
        if (candidate_ms) candidate_ms[cand] = ms / (float)reps;
        if (ms < best_ms) {
            best_ms = ms;
            best_shape = shape;
            best_cb = cands[cand].cb;
        }
    }
    // the last candidate: the graph of per-frame launches
    bool frames_win = false;
    if (st == PSFS_OK && cudaStreamSynchronize(b->user_stream) != cudaSuccess) st = fail(PSFS_ERR_CUDA, "batch autotune sync");
    if (st == PSFS_OK) st = batch_build_frames(b);
    if (st == PSFS_OK) {
        cudaError_t err = cudaGraphLaunch(b->exec, b->user_stream);   // warm-up
        if (err == cudaSuccess) err = cudaEventRecord(e0, b->user_stream);
        for (int r = 0; r < reps && err == cudaSuccess; ++r) err = cudaGraphLaunch(b->exec, b->user_stream);
        if (err == cudaSuccess) err = cudaEventRecord(e1, b->user_stream);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err != cudaSuccess) {
            st = fail_cuda(err, "batch autotune timing");
        } else {
            if (candidate_ms) candidate_ms[kBatchCandidates - 1] = ms / (float)reps;
            frames_win = ms < best_ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->cam_block = best_cb;
    if (st != PSFS_OK) return st;
    st = frames_win ? PSFS_OK : batch_build(b, best_shape);   // the frame-launch graph is built already
    if (st != PSFS_OK) return st;
    cudaMemsetAsync(b->d_words, 0, sizeof(uint32_t), b->user_stream);
    if (best) {
        best->lanes_x = best_shape.lx;
        best->warps = best_shape.wy;
        best->voxels_z = best_shape.tz;
        best->staged = 0;
        best->seq_likelihood_ctas = 0;
        best->frames_per_group = 0;
        best->cameras_per_block = best_cb;
        best->batch_launch = frames_win ? 1 : 0;
    }
    return PSFS_OK;
}

psfs_status psfs_batch_set_wait_limit(psfs_batch *b, uint64_t limit_ns, int32_t hold_frame)
{
    if (!b) return fail(PSFS_ERR_INVALID_ARG, "batch is NULL");
    if (limit_ns < 1000 || limit_ns > 10ull * kWaitNs)
        return fail(PSFS_ERR_INVALID_ARG, "wait limit outside [1 us, 10 s]");
    if (hold_frame < -1 || hold_frame >= (int32_t)b->frames.size())
        return fail(PSFS_ERR_INVALID_ARG, "hold_frame is not -1 or a frame of the batch");
    DeviceGuard guard(b->device);
    PSFS_CK(cudaStreamSynchronize(b->user_stream));
    b->wait_ns = limit_ns;
    b->hold_frame = hold_frame;
    return batch_build(b, b->shape);
}

void psfs_batch_destroy(psfs_batch *b) { batch_free(b); }

}  // extern "C"
