// api.cpp -- the C ABI of libbz.so (declared in include/bz.h).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "bz.h"
#include "kernels.h"

struct bz_ctx {
    std::atomic<int> refs;  // the context itself + each live mixture and swarm
    int device;
    bz_allocator alloc;
    bool custom_alloc;
    int sm_count;
    int smem_optin;
    // pinned host slots for swarm tallies, allocated in chunks and reused
    std::mutex pin_mu;
    std::vector<bz_tallies *> pin_free;
    std::vector<void *> pin_chunks;
    std::vector<std::pair<size_t, void *>> pin_blocks;  // free pinned blocks (capacity, pointer) for batches
    ~bz_ctx()
    {
        for (void *p : pin_chunks) cudaFreeHost(p);
        for (auto &b : pin_blocks) cudaFreeHost(b.second);
    }
};

struct bz_mixture {
    bz_ctx *ctx;
    bz::CompiledMixture cm;
    uint8_t *blob32, *blob64;
    size_t bytes32, bytes64;
    bool ch_smem32, ch_smem64;
};

struct bz_swarm {
    bz_ctx *ctx;
    bz_swarm_config cfg;
    cudaStream_t stream;
    uint8_t *mem;
    size_t bytes;
    bz::ParticlesDev p;
    uint32_t *err;
    bz_tallies *tallies_dev;
    bz_tallies *tallies_host;  // pinned
    cudaEvent_t done;
    cudaEvent_t ev[3];  // before the step kernel, after it, after the tallies
    uint64_t n;          // electrons (spawn mode: initial + created)
    uint64_t n_primary;
    uint64_t *bid;       // spawn mode: ids and birth times of the created electrons
    double *bt;
    bz::TallyArgs targs; // the tally kernels' arguments (group sums for merges)
};

struct bz_batch {
    bz_ctx *ctx;
    int32_t n;
    int precision;
    bool ch_smem, use_graph, ext, wide, bfield;
    size_t smem;
    int block, grid, n_tiles, max_tblocks;
    std::vector<uint64_t> n_el, id_offset;
    std::vector<bz::ParticlesDev> p;
    uint8_t *mem;
    size_t bytes;
    bz::RunArgs *desc;
    uint4 *tiles;
    unsigned int *tile_counter;
    uint32_t *errs;
    bz::TallyArgs *targs;
    bz_tallies *tallies_dev, *tallies_host;
    size_t tallies_cap;
    cudaStream_t cap;
    cudaGraph_t graph[2];      // [0]: counters + step kernel, [1]: tallies + copy to the host
    cudaGraphExec_t exec[2];
    cudaEvent_t ev[3], done;
    bool launched;
    std::vector<bz::TallyArgs> targs_host;  // per swarm (group sums for merges)
};

namespace {

thread_local std::string g_err;

bz_status fail(bz_status s, const std::string &msg)
{
    g_err = msg;
    return s;
}

bz_status cuda_fail(cudaError_t e, const char *where)
{
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    return BZ_ECUDA;
}

void *dev_alloc(bz_ctx *c, size_t bytes, cudaStream_t s)
{
    if (c->custom_alloc) return c->alloc.alloc(bytes, (void *)s, c->alloc.user);
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) return nullptr;
    return p;
}

void dev_free(bz_ctx *c, void *p, size_t bytes, cudaStream_t s)
{
    if (!p) return;
    if (c->custom_alloc) c->alloc.free(p, bytes, (void *)s, c->alloc.user);
    else cudaFreeAsync(p, s);
}

// Host-blocking copies that wait for nothing else.  cudaMemcpy runs on the
// legacy default stream, which first waits for all work queued there -- a
// caller's launch on that stream included, so a mixture compiled while the
// previous step runs would wait for it.  These copies take a non-blocking
// stream of their own and wait for that stream alone.
struct SyncCopies {
    cudaStream_t s = nullptr;
    cudaError_t e = cudaSuccess;
    SyncCopies() { e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking); }
    SyncCopies(const SyncCopies &) = delete;
    SyncCopies &operator=(const SyncCopies &) = delete;
    void add(void *dst, const void *src, size_t bytes, cudaMemcpyKind kind)
    {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, kind, s);
    }
    cudaError_t wait()
    {
        if (s) {
            const cudaError_t w = cudaStreamSynchronize(s);
            if (e == cudaSuccess) e = w;
        }
        return e;
    }
    ~SyncCopies()
    {
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    }
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Electrons per tile: ~n / (blocks x per_block), rounded up to a multiple of
// 256, within [256, 8192].
uint32_t tile_size_for(uint64_t n, uint64_t blocks, uint64_t per_block)
{
    uint64_t t = (n + blocks * per_block - 1) / (blocks * per_block);
    t = (t + 255) / 256 * 256;
    if (t < 256) t = 256;
    if (t > 8192) t = 8192;
    return (uint32_t)t;
}

// Tiles over the swarms in `order` (swarm index, electrons), in that order.
// Blocks take tiles in list order, so a launch ends when the last tiles
// taken end.  Tiles keep the full size while a quarter of an even share of
// the work left exceeds it, then shrink with the work left down to
// `min_tile` electrons (guided self-scheduling; the block's threads rounded
// up to a multiple of 256, so that the last tiles still give every lane an
// electron): a block that runs out of tiles waits at most about one short
// tile for the others, whatever the cost of the electrons that happen to
// come last.
void guided_tiles(const std::vector<std::pair<uint32_t, uint64_t>> &order, uint32_t tile, uint64_t blocks,
                  uint32_t min_tile, std::vector<uint4> *tiles)
{
    uint64_t left = 0;
    for (const auto &w : order) left += w.second;
    tiles->clear();
    for (const auto &w : order)
        for (uint64_t s0 = 0; s0 < w.second;) {
            uint64_t want = left / (4 * blocks);
            want = std::min<uint64_t>(std::max<uint64_t>((want + 255) / 256 * 256, min_tile), tile);
            const uint64_t c = std::min<uint64_t>(want, w.second - s0);
            tiles->push_back(make_uint4(w.first, (unsigned)s0, (unsigned)c, 0u));
            s0 += c;
            left -= c;
        }
}

void ctx_retain(bz_ctx *c) { c->refs.fetch_add(1); }

bz_tallies *pinned_slot(bz_ctx *c)
{
    std::lock_guard<std::mutex> lock(c->pin_mu);
    if (c->pin_free.empty()) {
        const int chunk = 256;
        void *p = nullptr;
        if (cudaMallocHost(&p, sizeof(bz_tallies) * chunk) != cudaSuccess) return nullptr;
        c->pin_chunks.push_back(p);
        for (int i = chunk - 1; i >= 0; --i) c->pin_free.push_back((bz_tallies *)p + i);
    }
    bz_tallies *t = c->pin_free.back();
    c->pin_free.pop_back();
    return t;
}

void pinned_release(bz_ctx *c, bz_tallies *t)
{
    if (!t) return;
    std::lock_guard<std::mutex> lock(c->pin_mu);
    c->pin_free.push_back(t);
}

// Pinned host block of at least `bytes` (power-of-two capacity), reused.
void *pinned_block(bz_ctx *c, size_t bytes, size_t *cap)
{
    size_t want = 4096;
    while (want < bytes) want <<= 1;
    {
        std::lock_guard<std::mutex> lock(c->pin_mu);
        for (size_t i = 0; i < c->pin_blocks.size(); ++i)
            if (c->pin_blocks[i].first == want) {
                void *p = c->pin_blocks[i].second;
                c->pin_blocks.erase(c->pin_blocks.begin() + i);
                *cap = want;
                return p;
            }
    }
    void *p = nullptr;
    if (cudaMallocHost(&p, want) != cudaSuccess) return nullptr;
    *cap = want;
    return p;
}

void pinned_block_release(bz_ctx *c, void *p, size_t cap)
{
    if (!p) return;
    std::lock_guard<std::mutex> lock(c->pin_mu);
    c->pin_blocks.emplace_back(cap, p);
}

// Host staging in page-locked memory from the context's pool, so that uploads
// start from pinned memory (one DMA) rather than from pageable vectors.  The
// block returns to the pool when the stage is destroyed: declare the stage
// before the SyncCopies whose copies read it, so that those copies are waited
// for first.
struct PinnedStage {
    bz_ctx *c;
    uint8_t *p = nullptr;
    size_t cap = 0, used = 0;
    PinnedStage(bz_ctx *ctx, size_t bytes) : c(ctx) { p = (uint8_t *)pinned_block(ctx, bytes, &cap); }
    PinnedStage(const PinnedStage &) = delete;
    PinnedStage &operator=(const PinnedStage &) = delete;
    ~PinnedStage() { pinned_block_release(c, p, cap); }
    // the pinned copy of `bytes` at `src`, or `src` itself if the pool had no room
    const void *put(const void *src, size_t bytes)
    {
        if (!p || used + bytes > cap) return src;
        uint8_t *d = p + used;
        memcpy(d, src, bytes);
        used = (used + bytes + 15) & ~(size_t)15;
        return d;
    }
};

void ctx_release(bz_ctx *c)
{
    if (c->refs.fetch_sub(1) == 1) delete c;
}

bz::Fields make_fields(const bz_swarm_config &cfg, double n_total)
{
    bz::Fields f;
    memset(&f, 0, sizeof f);
    const double E = cfg.e_over_n_Td * bz::kTownsend * n_total;
    f.a = bz::kQe * E / bz::kMe;
    f.has_b = cfg.b_T > 0.0 ? 1 : 0;
    f.b[0] = sin(cfg.b_angle_rad);
    f.b[1] = 0.0;
    f.b[2] = cos(cfg.b_angle_rad);
    f.w = bz::kQe * cfg.b_T / bz::kMe;
    if (f.has_b) {
        // E x B drift of the electron: (b x a z) / w
        f.vD[0] = f.a * f.b[1] / f.w;
        f.vD[1] = -f.a * f.b[0] / f.w;
        f.vD[2] = 0.0;
    }
    f.a_par = f.a * f.b[2];
    bz::Fields32 &g = f.f32;
    g.a = (float)f.a;
    g.b0 = (float)f.b[0];
    g.b1 = (float)f.b[1];
    g.b2 = (float)f.b[2];
    g.w = (float)f.w;
    g.inv_w = f.has_b ? (float)(1.0 / f.w) : 0.0f;
    g.vD0 = (float)f.vD[0];
    g.vD1 = (float)f.vD[1];
    g.vD2 = (float)f.vD[2];
    g.vDn = (float)sqrt(f.vD[0] * f.vD[0] + f.vD[1] * f.vD[1] + f.vD[2] * f.vD[2]);
    g.a_par = (float)f.a_par;
    g.Ke = (float)(0.5 * bz::kMe / bz::kQe);
    g.inv_a = f.a > 0.0 ? (float)(1.0 / f.a) : 0.0f;
    g.inv_apar = f.a_par != 0.0 ? (float)(1.0 / fabs(f.a_par)) : 0.0f;
    return f;
}

// The paper's adaptive trial frequencies (Sec. 6), run by the ADAPT
// instance of the step kernel.
bool adaptive(const bz_swarm_config *cfg)
{
    return cfg->trial_mode == BZ_TRIAL_VARIABLE || cfg->trial_mode == BZ_TRIAL_BINNED;
}

// Swarms that need the feature instance of the step kernel: the paper's
// adaptive trial frequencies, a mixture with an xi-form gas, or moving targets.
bool ext_instance(const bz_mixture *mix, const bz_swarm_config *cfg)
{
    return adaptive(cfg) || mix->cm.info.n_xi_gases > 0 || cfg->gas_temperature_K > 0.0;
}

bz_status validate_config(const bz_swarm_config *cfg)
{
    if (!cfg) return fail(BZ_EINVAL, "null configuration");
    if (cfg->precision != 32 && cfg->precision != 64) return fail(BZ_EINVAL, "precision must be 32 or 64");
    if (cfg->n_electrons < 1) return fail(BZ_EINVAL, "n_electrons must be >= 1");
    if (cfg->real_collisions < 1) return fail(BZ_EINVAL, "real_collisions must be >= 1");
    if (!(cfg->e_over_n_Td >= 0.0) || !isfinite(cfg->e_over_n_Td)) return fail(BZ_EINVAL, "bad E/N");
    if (!(cfg->b_T >= 0.0) || !isfinite(cfg->b_T) || !isfinite(cfg->b_angle_rad)) return fail(BZ_EINVAL, "bad B");
    if (cfg->trial_mode < BZ_TRIAL_LAZY || cfg->trial_mode > BZ_TRIAL_BINNED) return fail(BZ_EINVAL, "bad trial mode");
    if (adaptive(cfg)) {
        if (!(cfg->zeta >= 0.0) || !isfinite(cfg->zeta)) return fail(BZ_EINVAL, "zeta must be finite and >= 0");
        if (cfg->grace < 1) return fail(BZ_EINVAL, "grace must be >= 1");
        if (cfg->trial_mode == BZ_TRIAL_BINNED && (cfg->bins_per_decade < 1 || cfg->bins_per_decade > 32 ||
                                                   (cfg->bins_per_decade & (cfg->bins_per_decade - 1))))
            return fail(BZ_EINVAL, "bins_per_decade must be 1, 2, 4, 8, 16 or 32");
        if (cfg->spawn) return fail(BZ_EINVAL, "spawn mode runs with the lazy, fixed or windowed trial frequency");
    }
    if (!(cfg->window_c >= 0.0) || !isfinite(cfg->window_c)) return fail(BZ_EINVAL, "window_c must be >= 0");
    if (cfg->trial_mode == BZ_TRIAL_FIXED && !(cfg->nu_trial > 0.0)) return fail(BZ_EINVAL, "fixed mode needs nu_trial > 0");
    if (!(cfg->eps0_mean_eV >= 0.0) || !isfinite(cfg->eps0_mean_eV)) return fail(BZ_EINVAL, "bad eps0_mean_eV");
    if (!(cfg->t_end_s >= 0.0) || !isfinite(cfg->t_end_s)) return fail(BZ_EINVAL, "bad t_end_s");
    if (!(cfg->gas_temperature_K >= 0.0) || !isfinite(cfg->gas_temperature_K))
        return fail(BZ_EINVAL, "gas_temperature_K must be finite and >= 0");
    if (!isfinite(cfg->spawn_wait_s) || cfg->spawn_wait_s > 3600.0)
        return fail(BZ_EINVAL, "spawn_wait_s must be finite and at most 3600");
    if (cfg->hold_pending && !cfg->spawn) return fail(BZ_EINVAL, "hold_pending applies to spawn mode only");
    if (!isfinite(cfg->stage_wait_s) || cfg->stage_wait_s > 3600.0)
        return fail(BZ_EINVAL, "stage_wait_s must be finite and at most 3600");
    if (cfg->hold_stage > 1) return fail(BZ_EINVAL, "hold_stage must be 0 or 1");
    if (cfg->max_trials > 0xFFFFFFFFull) return fail(BZ_EINVAL, "max_trials must fit 32 bits");
    if (cfg->block_threads != 0 && cfg->block_threads != 128 && cfg->block_threads != 256 &&
        cfg->block_threads != 384 && cfg->block_threads != 768)
        return fail(BZ_EINVAL, "block_threads must be 0, 128, 256, 384 or 768");
    if (cfg->block_threads != 0 && cfg->block_threads != 256 && (cfg->precision != 32 || cfg->spawn))
        return fail(BZ_EINVAL, "blocks of 128, 384 or 768 threads run FP32 swarms without spawn mode only");
    if (cfg->blocks_per_sm < 0) return fail(BZ_EINVAL, "blocks_per_sm must be >= 0");
    if (cfg->spawn != 0 && cfg->spawn != 1) return fail(BZ_EINVAL, "spawn must be 0 or 1");
    if (cfg->spawn && cfg->pop_cap && cfg->pop_cap < cfg->n_electrons)
        return fail(BZ_EINVAL, "pop_cap below the number of initial electrons");
    return BZ_OK;
}

// Fills the kernel arguments common to swarm runs and replays.
bz_status prepare_run(const bz_mixture *mix, const bz_swarm_config *cfg, bz::RunArgs *a, bool *ch_smem)
{
    memset(a, 0, sizeof *a);
    const bool p64 = cfg->precision == 64;
    a->blob = p64 ? mix->blob64 : mix->blob32;
    a->lay = p64 ? mix->cm.lay64 : mix->cm.lay32;
    *ch_smem = p64 ? mix->ch_smem64 : mix->ch_smem32;
    a->stage_bytes = *ch_smem ? a->lay.stage_all : a->lay.stage_tables;
    if ((int)a->stage_bytes > mix->ctx->smem_optin - 1024)
        return fail(BZ_EBUDGET, "mixture tables exceed the shared memory of one block");
    a->key0 = (uint32_t)cfg->seed;
    a->key1 = (uint32_t)(cfg->seed >> 32);
    for (uint32_t r = 0; r < 10; ++r) {  // Philox round keys, read by the step instead of stepped
        a->rk[2 * r] = a->key0 + r * 0x9E3779B9u;
        a->rk[2 * r + 1] = a->key1 + r * 0xBB67AE85u;
    }
    a->id_offset = cfg->id_offset;
    a->n = cfg->n_electrons;
    a->I = cfg->real_collisions;
    a->fixed = cfg->trial_mode == BZ_TRIAL_FIXED;
    a->attach_keep = cfg->attach_keep_state != 0;
    a->nu0 = (cfg->nu_trial > 0.0) ? cfg->nu_trial : mix->cm.nu_trial;
    a->eps0_mean = cfg->eps0_mean_eV;
    a->spawn_wait_ns = (uint64_t)((cfg->spawn_wait_s > 0.0 ? cfg->spawn_wait_s : 60.0) * 1e9);
    a->stage_wait_ns = (uint64_t)((cfg->stage_wait_s > 0.0 ? cfg->stage_wait_s : 10.0) * 1e9);
    a->stage_hold = cfg->hold_stage;
    a->v0_scale = sqrt((2.0 / 3.0) * cfg->eps0_mean_eV * bz::kQe / bz::kMe);
    a->v0_scale32 = (float)a->v0_scale;
    a->nu0_32 = (float)a->nu0;
    a->t_end = cfg->t_end_s;
    a->max_trials = cfg->max_trials ? cfg->max_trials : 0x7FFFFFFFull;
    a->window = cfg->trial_mode == BZ_TRIAL_WINDOW;
    a->win_c = (float)(cfg->window_c > 0.0 ? cfg->window_c : 2.0);
    a->nu_floor = 1e-9 * mix->cm.nu_max;
    a->f = make_fields(*cfg, mix->cm.n_total);
    a->tf = cfg->trial_mode == BZ_TRIAL_VARIABLE ? bz::TF_VARIABLE
            : cfg->trial_mode == BZ_TRIAL_BINNED ? bz::TF_BINNED : bz::TF_NONE;
    a->tf_zeta1 = 1.0 + cfg->zeta;
    a->kT_m = 1.380649e-23 * cfg->gas_temperature_K / bz::kMe;  // Boltzmann constant [J/K]
    a->kT_m32 = (float)a->kT_m;
    a->thermal = a->kT_m > 0.0;
    // the adaptive nu' is never below nu at the lowest table energy (nu
    // vanishes at rest, and the tables say nothing below their first point)
    if (a->tf != bz::TF_NONE) a->nu_floor = std::max(a->nu_floor, a->lay.nu_first);
    a->nu_floor32 = (float)a->nu_floor;
    a->timed = a->t_end > 0.0;
    a->tf_grace = cfg->grace;
    a->tf_B = cfg->bins_per_decade;
    if (a->tf == bz::TF_BINNED && (a->lay.bins_per_decade % cfg->bins_per_decade) != 0)
        return fail(BZ_EINVAL, "bins_per_decade must divide the mixture's compiled bins per decade");
    return BZ_OK;
}

}  // namespace

void bz::set_last_error(const std::string &msg) { g_err = msg; }
int bz::ctx_device(const bz_ctx *ctx) { return ctx->device; }
bz_status bz::check_config(const bz_swarm_config *cfg) { return validate_config(cfg); }
bool bz::needs_feature_instance(const bz_mixture *mix, const bz_swarm_config *cfg) { return ext_instance(mix, cfg); }
bool bz::stages_channels(const bz_mixture *mix, int precision) { return precision == 64 ? mix->ch_smem64 : mix->ch_smem32; }

extern "C" {

const char *bz_last_error(void) { return g_err.c_str(); }
int bz_abi_version(void) { return BZ_ABI_VERSION; }

bz_status bz_create(int device, const bz_allocator *alloc, bz_ctx **out)
{
    if (!out) return fail(BZ_EINVAL, "null output");
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= n) return fail(BZ_EINVAL, "no such CUDA device");
    if ((e = cudaSetDevice(device)) != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    if (alloc && (!alloc->alloc || !alloc->free)) return fail(BZ_EINVAL, "allocator needs alloc and free");
    bz_ctx *c = new (std::nothrow) bz_ctx();
    if (!c) return fail(BZ_ENOMEM, "host allocation");
    c->refs.store(1);
    c->device = device;
    c->custom_alloc = alloc != nullptr;
    if (alloc) c->alloc = *alloc;
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    *out = c;
    return BZ_OK;
}

void bz_destroy(bz_ctx *ctx)
{
    if (ctx) ctx_release(ctx);
}

bz_status bz_create_gas_mixture(bz_ctx *ctx, const bz_gas *gases, int32_t n_gases, const bz_mixture_opts *opts,
                                bz_mixture **out)
{
    if (!ctx || !out) return fail(BZ_EINVAL, "null argument");
    *out = nullptr;
    bz_mixture *m = new (std::nothrow) bz_mixture();
    if (!m) return fail(BZ_ENOMEM, "host allocation");
    m->ctx = ctx;
    std::string err;
    bz_status st = bz::compile_mixture(gases, n_gases, opts, &m->cm, &err);
    if (st != BZ_OK) {
        delete m;
        return fail(st, err);
    }
    cudaSetDevice(ctx->device);
    m->bytes32 = m->cm.blob32.size();
    m->bytes64 = m->cm.blob64.size();
    PinnedStage stage(ctx, m->bytes32 + m->bytes64 + 32);
    SyncCopies up;
    // the library's own pool allocates in the order of the copy stream; a
    // caller's allocator takes its usual stream (the tables are freed only
    // after a device-wide synchronisation)
    const cudaStream_t as = ctx->custom_alloc ? (cudaStream_t)0 : up.s;
    m->blob32 = (uint8_t *)dev_alloc(ctx, m->bytes32, as);
    m->blob64 = (uint8_t *)dev_alloc(ctx, m->bytes64, as);
    if (!m->blob32 || !m->blob64) {
        up.wait();
        dev_free(ctx, m->blob32, m->bytes32, as);
        dev_free(ctx, m->blob64, m->bytes64, as);
        delete m;
        return fail(BZ_ENOMEM, "device allocation of the mixture tables");
    }
    up.add(m->blob32, stage.put(m->cm.blob32.data(), m->bytes32), m->bytes32, cudaMemcpyHostToDevice);
    up.add(m->blob64, stage.put(m->cm.blob64.data(), m->bytes64), m->bytes64, cudaMemcpyHostToDevice);
    cudaError_t e = up.wait();
    if (e != cudaSuccess) {
        dev_free(ctx, m->blob32, m->bytes32, 0);
        dev_free(ctx, m->blob64, m->bytes64, 0);
        delete m;
        return cuda_fail(e, "copy of the mixture tables");
    }
    const int mode = opts ? opts->channels_in_smem : -1;
    // channel values go to shared memory when the whole staged blob fits the
    // budget the tables were compiled for (three FP32 blocks per SM)
    int budget = (opts && opts->smem_budget > 0) ? opts->smem_budget : (int)bz::kStageBudget32;
    if (budget > ctx->smem_optin - 1024) budget = ctx->smem_optin - 1024;
    int budget64 = std::min((int)bz::kStageBudget64, ctx->smem_optin - 1024);
    m->ch_smem32 = mode == 1 ? true : mode == 0 ? false : (int)m->cm.lay32.stage_all <= budget;
    m->ch_smem64 = mode == 1 ? true : mode == 0 ? false : (int)m->cm.lay64.stage_all <= budget64;
    if (m->ch_smem32 && (int)m->cm.lay32.stage_all > ctx->smem_optin - 1024) m->ch_smem32 = false;
    if (m->ch_smem64 && (int)m->cm.lay64.stage_all > ctx->smem_optin - 1024) m->ch_smem64 = false;
    m->cm.info.channels_in_smem = m->ch_smem32 ? 1 : 0;
    m->cm.info.smem_bytes = (int32_t)(m->ch_smem32 ? m->cm.lay32.stage_all : m->cm.lay32.stage_tables);
    m->cm.info.table_bytes = (int32_t)(m->bytes32 + m->bytes64);
    ctx_retain(ctx);
    *out = m;
    return BZ_OK;
}

void bz_destroy_mixture(bz_mixture *mix)
{
    if (!mix) return;
    cudaSetDevice(mix->ctx->device);
    cudaDeviceSynchronize();
    dev_free(mix->ctx, mix->blob32, mix->bytes32, 0);
    dev_free(mix->ctx, mix->blob64, mix->bytes64, 0);
    bz_ctx *ctx = mix->ctx;
    delete mix;
    ctx_release(ctx);
}

bz_status bz_mixture_get_info(const bz_mixture *mix, bz_mixture_info *out)
{
    if (!mix || !out) return fail(BZ_EINVAL, "null argument");
    *out = mix->cm.info;
    return BZ_OK;
}

bz_status bz_mixture_compile_info(const bz_gas *gases, int32_t n_gases, const bz_mixture_opts *opts,
                                  bz_mixture_info *out)
{
    if (!out) return fail(BZ_EINVAL, "null argument");
    bz::CompiledMixture cm;
    std::string err;
    bz_status st = bz::compile_mixture(gases, n_gases, opts, &cm, &err);
    if (st != BZ_OK) return fail(st, err);
    *out = cm.info;
    return BZ_OK;
}

void bz_config_defaults(bz_swarm_config *cfg)
{
    if (!cfg) return;
    memset(cfg, 0, sizeof *cfg);
    cfg->n_electrons = 10000;
    cfg->real_collisions = 1000;
    cfg->precision = 32;
    cfg->trial_mode = BZ_TRIAL_LAZY;
    cfg->eps0_mean_eV = 0.1;
    cfg->seed = 1901081400ull;
    cfg->zeta = 0.25;
    cfg->grace = 5000;
    cfg->bins_per_decade = 8;
}

bz_status bz_set_fields(bz_swarm_config *cfg, double e_over_n_Td, double b_T, double b_angle_rad)
{
    if (!cfg) return fail(BZ_EINVAL, "null configuration");
    if (!(e_over_n_Td >= 0.0) || !isfinite(e_over_n_Td)) return fail(BZ_EINVAL, "E/N must be finite and >= 0");
    if (!(b_T >= 0.0) || !isfinite(b_T)) return fail(BZ_EINVAL, "|B| must be finite and >= 0");
    if (!isfinite(b_angle_rad)) return fail(BZ_EINVAL, "B angle must be finite");
    cfg->e_over_n_Td = e_over_n_Td;
    cfg->b_T = b_T;
    cfg->b_angle_rad = b_angle_rad;
    return BZ_OK;
}

bz_status bz_run_swarm(bz_ctx *ctx, const bz_mixture *mix, const bz_swarm_config *cfg, void *stream,
                       bz_swarm **out)
{
    if (!ctx || !mix || !out) return fail(BZ_EINVAL, "null argument");
    *out = nullptr;
    bz_status st = validate_config(cfg);
    if (st != BZ_OK) return st;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    bz::RunArgs a;
    bool ch_smem;
    if ((st = prepare_run(mix, cfg, &a, &ch_smem)) != BZ_OK) return st;
    const uint64_t n = cfg->n_electrons;
    const bool spawn = cfg->spawn != 0;
    const uint64_t cap = spawn ? (cfg->pop_cap ? cfg->pop_cap : 64 * n) : n;  // electron slots
    if (cap > 0xFFFFFFFFull) return fail(BZ_EINVAL, "a swarm holds at most 2^32-1 electrons");
    const int block = cfg->block_threads ? cfg->block_threads : 256;
    if (block != 256 && ext_instance(mix, cfg))
        return fail(BZ_EINVAL, "blocks of 128, 384 or 768 threads run the lean step kernel only (no VARIABLE / "
                               "BINNED trial frequency, no xi-form gases)");
    const bool bfield = cfg->b_T > 0.0;
    // the 4-block build: for every mixture without B; with B (more registers
    // live, more spills at 64) only for one gas; blocks of 256 threads only
    const bool wide = block == 256 && (!bfield || mix->cm.info.n_gases == 1);
    int bps = spawn ? bz::spawn_occupancy(cfg->precision, ch_smem, ext_instance(mix, cfg), wide, bfield, block,
                                          a.stage_bytes)
                    : bz::batch_occupancy(cfg->precision, ch_smem, ext_instance(mix, cfg), wide, bfield, block,
                                          a.stage_bytes);
    if (bps < 0) return cuda_fail((cudaError_t)(-bps), "occupancy of the step kernel");
    if (bps < 1) return fail(BZ_ECUDA, "step kernel cannot be resident with these tables");
    if (cfg->blocks_per_sm > 0 && cfg->blocks_per_sm < bps) bps = cfg->blocks_per_sm;
    const uint64_t grid64 = (uint64_t)ctx->sm_count * bps;
    const int tblocks = bz::tally_blocks(cap, ctx->sm_count);

    bz_swarm *s = new (std::nothrow) bz_swarm();
    if (!s) return fail(BZ_ENOMEM, "host allocation");
    s->ctx = ctx;
    ctx_retain(ctx);
    s->cfg = *cfg;
    s->stream = (cudaStream_t)stream;
    s->n = n;
    s->n_primary = n;
    // one device block: particle outputs, counters and flags, birth records, tally scratch
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    const uint64_t m = cap;
    const size_t o_x = take(8 * m), o_y = take(8 * m), o_z = take(8 * m), o_t = take(8 * m);
    const size_t o_se = take(8 * m), o_se2 = take(8 * m);
    const size_t o_vx = take(4 * m), o_vy = take(4 * m), o_vz = take(4 * m), o_nup = take(4 * m);
    const size_t o_u[7] = {take(4 * m), take(4 * m), take(4 * m), take(4 * m), take(4 * m), take(4 * m), take(4 * m)};
    // tile counter, error word, capped counter; spawn mode: electrons, pending, ticket
    const size_t o_ctr = take(48);
    const uint64_t nb = spawn ? cap - n : 0;
    const size_t o_bt = take(8 * nb), o_bid = take(8 * nb), o_bv = take(24 * nb);
    const size_t o_p1 = take(sizeof(double) * tblocks * bz::kGroups * bz::kQ1);
    const size_t o_p2 = take(sizeof(double) * tblocks * bz::kGroups * bz::kQ2);
    const size_t o_gs = take(sizeof(double) * (bz::kGroups * (bz::kQ1 + bz::kQ2) + 8));
    const size_t o_tal = take(sizeof(bz_tallies));
    s->bytes = off;
    s->mem = (uint8_t *)dev_alloc(ctx, s->bytes, s->stream);
    if (!s->mem) {
        delete s;
        ctx_release(ctx);
        return fail(BZ_ENOMEM, "device allocation of the swarm state");
    }
    uint8_t *M = s->mem;
    s->p = bz::ParticlesDev{(double *)(M + o_x), (double *)(M + o_y), (double *)(M + o_z), (double *)(M + o_t),
                            (double *)(M + o_se), (double *)(M + o_se2), (float *)(M + o_vx), (float *)(M + o_vy),
                            (float *)(M + o_vz), (float *)(M + o_nup), (uint32_t *)(M + o_u[0]),
                            (uint32_t *)(M + o_u[1]), (uint32_t *)(M + o_u[2]), (uint32_t *)(M + o_u[3]),
                            (uint32_t *)(M + o_u[4]), (uint32_t *)(M + o_u[5]), (uint32_t *)(M + o_u[6])};
    unsigned int *counter = (unsigned int *)(M + o_ctr);
    s->err = (uint32_t *)(M + o_ctr + 8);
    unsigned int *n_capped = (unsigned int *)(M + o_ctr + 12);
    unsigned long long *n_total = (unsigned long long *)(M + o_ctr + 16);
    unsigned long long *pending = (unsigned long long *)(M + o_ctr + 24);
    unsigned long long *ticket = (unsigned long long *)(M + o_ctr + 32);
    s->bt = (double *)(M + o_bt);
    s->bid = (uint64_t *)(M + o_bid);
    s->tallies_dev = (bz_tallies *)(M + o_tal);
    s->tallies_host = pinned_slot(ctx);
    if (!s->tallies_host) e = cudaErrorMemoryAllocation;
    else e = cudaEventCreateWithFlags(&s->done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        dev_free(ctx, s->mem, s->bytes, s->stream);
        pinned_release(ctx, s->tallies_host);
        if (s->done) cudaEventDestroy(s->done);
        delete s;
        ctx_release(ctx);
        return cuda_fail(e, "swarm set-up");
    }
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaEventCreate(&s->ev[i]);
    if (e == cudaSuccess) e = cudaMemsetAsync(M + o_ctr, 0, 48, s->stream);
    a.counter = nullptr;
    a.err = s->err;
    a.out = s->p;
    a.spawn = spawn ? 1 : 0;
    a.n_primary = n;
    a.cap = cap;
    a.n_total = n_total;
    a.pending = pending;
    a.n_capped = n_capped;
    a.bt = s->bt;
    a.bid = s->bid;
    a.bvx = (double *)(M + o_bv);
    a.bvy = a.bvx + nb;
    a.bvz = a.bvy + nb;
    // spawn mode: electrons, pending (plus the electrons a test holds pending)
    const unsigned long long init[2] = {n, n + cfg->hold_pending};
    if (spawn) {
        // unpublished birth records read as id 0
        a.counter = ticket;
        if (e == cudaSuccess && nb) e = cudaMemsetAsync(s->bid, 0, 8 * nb, s->stream);
        // staged in the swarm's pinned tally slot (its tallies arrive there
        // later in stream order): a copy from pageable memory would first wait
        // for the stream's earlier work
        static_assert(sizeof(bz_tallies) >= sizeof init, "tally slot too small");
        memcpy(s->tallies_host, init, sizeof init);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(n_total, s->tallies_host, sizeof init, cudaMemcpyHostToDevice, s->stream);
    }
    if (e == cudaSuccess) e = cudaEventRecord(s->ev[0], s->stream);
    if (!spawn) {
        // tiles over all slots, one launch
        bz::BatchArgs ba;
        memset(&ba, 0, sizeof ba);
        ba.tile_counter = counter;
        ba.single = a;
        // equal tiles computed in the kernel: a tile list would have to be
        // copied from pageable memory, which waits for the stream's earlier work
        // (at least one electron per thread of a block)
        const uint32_t tile = std::max<uint32_t>(tile_size_for(n, grid64, 8), (uint32_t)(block + 255) / 256 * 256);
        const uint64_t n_tiles = (n + tile - 1) / tile;
        ba.n_tiles = (int32_t)n_tiles;
        ba.tile_size = tile;
        ba.slot_lo = 0;
        const int grid = (int)(grid64 < n_tiles ? grid64 : n_tiles);
        if (e == cudaSuccess && n_tiles > 0)
            e = bz::launch_batch(cfg->precision, ch_smem, ext_instance(mix, cfg), wide, bfield, ba, a.stage_bytes,
                                 grid, block, s->stream);
    } else {
        // every electron, created ones included, in one persistent launch:
        // a lane per electron of the population cap (at least a block per
        // SM).  Fewer blocks leave room for concurrent launches but made a
        // 1e5-cap avalanche 50 % slower and served requests slower overall.
        uint64_t want = (cap + block - 1) / block;
        if (want < (uint64_t)ctx->sm_count) want = ctx->sm_count;
        const int grid = (int)(grid64 < want ? grid64 : want);
        if (e == cudaSuccess) e = bz::launch_spawn(cfg->precision, ch_smem, ext_instance(mix, cfg), wide, bfield, a,
                                                  a.stage_bytes, grid, block, s->stream);
    }
    if (e == cudaSuccess) e = cudaEventRecord(s->ev[1], s->stream);
    bz::TallyArgs t;
    memset(&t, 0, sizeof t);
    t.x = s->p.x; t.y = s->p.y; t.z = s->p.z; t.t = s->p.t; t.se = s->p.se; t.se2 = s->p.se2;
    t.n_real = s->p.n_real; t.n_null = s->p.n_null; t.n_fail = s->p.n_fail; t.n_ion = s->p.n_ion;
    t.n_att = s->p.n_att; t.status = s->p.status;
    t.steps = s->p.steps;
    t.n = spawn ? cap : n;
    t.n_dev = spawn ? n_total : nullptr;
    t.n_primary = n;
    t.ids = spawn ? s->bid : nullptr;
    t.capped = spawn ? n_capped : nullptr;
    t.id_offset = cfg->id_offset;
    t.part1 = (double *)(M + o_p1);
    t.part2 = (double *)(M + o_p2);
    t.gsum = (double *)(M + o_gs);
    t.blocks = tblocks;
    t.E_V_m = cfg->e_over_n_Td * bz::kTownsend * mix->cm.n_total;
    t.n_total = mix->cm.n_total;
    t.nu_trial = a.nu0;
    t.err = s->err;
    t.out = s->tallies_dev;
    s->targs = t;
    if (e == cudaSuccess) e = bz::launch_tallies(t, s->stream);
    if (e == cudaSuccess) e = cudaEventRecord(s->ev[2], s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->tallies_host, s->tallies_dev, sizeof(bz_tallies), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaEventRecord(s->done, s->stream);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(s->stream);
        bz_destroy_swarm(s);
        return cuda_fail(e, "swarm launch");
    }
    *out = s;
    return BZ_OK;
}

static bz_status finish_tallies(bz_swarm *sw, bz_tallies *out)
{
    *out = *sw->tallies_host;
    if (out->error_flags & BZ_ERR_STAGE_TIMEOUT) return fail(BZ_ETIMEOUT, "table staging timed out");
    if (out->error_flags & BZ_ERR_SPAWN_WAIT) return fail(BZ_ETIMEOUT, "spawn mode: a wait for created electrons gave up");
    if (out->error_flags & BZ_ERR_TRIAL) return fail(BZ_ETRIAL, "trial frequency exceeded (fixed mode, or a binned retry that failed again)");
    return BZ_OK;
}

bz_status bz_read_tallies(bz_swarm *sw, bz_tallies *out)
{
    if (!sw || !out) return fail(BZ_EINVAL, "null argument");
    cudaError_t e = cudaEventSynchronize(sw->done);
    if (e != cudaSuccess) return cuda_fail(e, "swarm");
    return finish_tallies(sw, out);
}

bz_status bz_query_tallies(bz_swarm *sw, bz_tallies *out)
{
    if (!sw || !out) return fail(BZ_EINVAL, "null argument");
    cudaError_t e = cudaEventQuery(sw->done);
    if (e == cudaErrorNotReady) return BZ_ENOTREADY;
    if (e != cudaSuccess) return cuda_fail(e, "swarm");
    return finish_tallies(sw, out);
}

// Electrons in a finished swarm (spawn mode: the primaries and the created ones).
static uint64_t swarm_count(const bz_swarm *sw)
{
    if (!sw->cfg.spawn) return sw->n;
    return sw->n_primary + sw->tallies_host->n_spawned;
}

bz_status bz_read_particles(bz_swarm *sw, const bz_particles *o)
{
    if (!sw || !o) return fail(BZ_EINVAL, "null argument");
    cudaError_t e = cudaEventSynchronize(sw->done);
    if (e != cudaSuccess) return cuda_fail(e, "swarm");
    const size_t n = sw->n = swarm_count(sw);
    struct { void *dst; const void *src; size_t bytes; } cp[] = {
        {o->x, sw->p.x, 8 * n}, {o->y, sw->p.y, 8 * n}, {o->z, sw->p.z, 8 * n}, {o->t, sw->p.t, 8 * n},
        {o->sum_e, sw->p.se, 8 * n}, {o->sum_e2, sw->p.se2, 8 * n}, {o->vx, sw->p.vx, 4 * n},
        {o->vy, sw->p.vy, 4 * n}, {o->vz, sw->p.vz, 4 * n}, {o->nu_p, sw->p.nup, 4 * n},
        {o->n_real, sw->p.n_real, 4 * n}, {o->n_null, sw->p.n_null, 4 * n}, {o->n_fail, sw->p.n_fail, 4 * n},
        {o->n_ion, sw->p.n_ion, 4 * n}, {o->n_att, sw->p.n_att, 4 * n}, {o->steps, sw->p.steps, 4 * n},
        {o->status, sw->p.status, 4 * n}};
    SyncCopies rd;
    for (auto &c : cp)
        if (c.dst) rd.add(c.dst, c.src, c.bytes, cudaMemcpyDeviceToHost);
    const uint64_t np = sw->n_primary < n ? sw->n_primary : n;
    if (o->id) {
        for (uint64_t i = 0; i < np; ++i) o->id[i] = sw->cfg.id_offset + i;
        if (n > np) rd.add(o->id + np, sw->bid, 8 * (n - np), cudaMemcpyDeviceToHost);
    }
    if (o->t_birth) {
        for (uint64_t i = 0; i < np; ++i) o->t_birth[i] = 0.0;
        if (n > np) rd.add(o->t_birth + np, sw->bt, 8 * (n - np), cudaMemcpyDeviceToHost);
    }
    if ((e = rd.wait()) != cudaSuccess) return cuda_fail(e, "copy of particle state");
    return BZ_OK;
}

bz_status bz_swarm_size(bz_swarm *sw, uint64_t *n)
{
    if (!sw || !n) return fail(BZ_EINVAL, "null argument");
    cudaError_t e = cudaEventSynchronize(sw->done);
    if (e != cudaSuccess) return cuda_fail(e, "swarm");
    *n = sw->n = swarm_count(sw);
    return BZ_OK;
}

void bz_destroy_swarm(bz_swarm *sw)
{
    if (!sw) return;
    cudaSetDevice(sw->ctx->device);
    if (sw->done) cudaEventSynchronize(sw->done);
    else cudaStreamSynchronize(sw->stream);
    dev_free(sw->ctx, sw->mem, sw->bytes, sw->stream);
    pinned_release(sw->ctx, sw->tallies_host);
    if (sw->done) cudaEventDestroy(sw->done);
    for (int i = 0; i < 3; ++i)
        if (sw->ev[i]) cudaEventDestroy(sw->ev[i]);
    bz_ctx *ctx = sw->ctx;
    delete sw;
    ctx_release(ctx);
}

bz_status bz_swarm_timing(bz_swarm *sw, double *step_ms, double *tally_ms)
{
    if (!sw) return fail(BZ_EINVAL, "null argument");
    cudaError_t e = cudaEventSynchronize(sw->done);
    float a = 0.f, b = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&a, sw->ev[0], sw->ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&b, sw->ev[1], sw->ev[2]);
    if (e != cudaSuccess) return cuda_fail(e, "swarm timing");
    if (step_ms) *step_ms = a;
    if (tally_ms) *tally_ms = b;
    return BZ_OK;
}

// ---------------------------------------------------------------------------
// Batches
// ---------------------------------------------------------------------------
// part 0: counters and the step kernel; part 1: tallies and their copy to the host
static cudaError_t batch_part(bz_batch *b, int part, cudaStream_t s)
{
    cudaError_t e;
    if (part == 0) {
        e = cudaMemsetAsync(b->tile_counter, 0, sizeof(unsigned int) * (2 + b->n), s);
        bz::BatchArgs a;
        memset(&a, 0, sizeof a);
        a.desc = b->desc;
        a.tiles = b->tiles;
        a.n_tiles = b->n_tiles;
        a.tile_counter = b->tile_counter;
        if (e == cudaSuccess) e = bz::launch_batch(b->precision, b->ch_smem, b->ext, b->wide, b->bfield, a, b->smem, b->grid, b->block, s);
        return e;
    }
    e = bz::launch_tallies_multi(b->targs, b->n, b->max_tblocks, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->tallies_host, b->tallies_dev, sizeof(bz_tallies) * b->n, cudaMemcpyDeviceToHost, s);
    return e;
}

static bz_status batch_sequence(bz_batch *b, cudaStream_t s)
{
    cudaError_t e = cudaEventRecord(b->ev[0], s);
    for (int part = 0; part < 2 && e == cudaSuccess; ++part) {
        e = b->use_graph ? cudaGraphLaunch(b->exec[part], s) : batch_part(b, part, s);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev[1 + part], s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "batch launch");
    return BZ_OK;
}

bz_status bz_create_batch(bz_ctx *ctx, int32_t n, const bz_mixture *const *mixtures, const bz_swarm_config *cfgs,
                          const bz_batch_opts *opts, bz_batch **out)
{
    if (!ctx || !out || !mixtures || !cfgs) return fail(BZ_EINVAL, "null argument");
    *out = nullptr;
    if (n < 1) return fail(BZ_EINVAL, "a batch needs at least one swarm");
    // the tally kernels take one grid row per swarm
    if (n > 65535) return fail(BZ_EINVAL, "a batch holds at most 65535 swarms");
    const int precision = cfgs[0].precision;
    for (int i = 0; i < n; ++i) {
        bz_status st = validate_config(&cfgs[i]);
        if (st != BZ_OK) return st;
        if (!mixtures[i] || !mixtures[0]) return fail(BZ_EINVAL, "null mixture");
        if (cfgs[i].precision != precision) return fail(BZ_EINVAL, "all swarms of a batch need the same precision");
        if (cfgs[i].spawn) return fail(BZ_EINVAL, "spawn-mode swarms run through bz_run_swarm");
        if (ext_instance(mixtures[i], &cfgs[i]) != ext_instance(mixtures[0], &cfgs[0]))
            return fail(BZ_EINVAL, "a batch holds either swarms with VARIABLE / BINNED trial frequencies or xi-form "
                                   "gases, or swarms with neither");
        if (cfgs[i].n_electrons > 0xFFFFFFFFull) return fail(BZ_EINVAL, "a batched swarm holds at most 2^32-1 electrons");
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    bz_batch *b = new (std::nothrow) bz_batch();
    if (!b) return fail(BZ_ENOMEM, "host allocation");
    b->ctx = ctx;
    b->n = n;
    b->precision = precision;
    b->ext = ext_instance(mixtures[0], &cfgs[0]);
    b->bfield = false;  // the lean build without the field's paths when no swarm has B
    for (int i = 0; i < n; ++i) b->bfield = b->bfield || cfgs[i].b_T > 0.0;
    b->block = (opts && opts->block_threads > 0) ? opts->block_threads : 256;
    if (b->block != 256 && b->block != 128 && b->block != 384 && b->block != 768) {
        delete b;
        return fail(BZ_EINVAL, "block_threads must be 0, 128, 256, 384 or 768");
    }
    if (b->block != 256 && (precision != 32 || b->ext)) {
        delete b;
        return fail(BZ_EINVAL, "blocks of 128, 384 or 768 threads run the lean FP32 step kernel only");
    }
    // the 4-block build: without B, or when every mixture has one gas; blocks of 256 threads only
    b->wide = b->block == 256;
    for (int i = 0; i < n; ++i) b->wide = b->wide && (!b->bfield || mixtures[i]->cm.info.n_gases == 1);
    b->use_graph = opts ? opts->use_graph != 0 : true;
    // tables of every mixture must fit; channel tables go to shared memory only if all fit
    b->ch_smem = true;
    std::vector<bz::RunArgs> desc(n);
    for (int i = 0; i < n; ++i) {
        bool ch;
        bz_status st = prepare_run(mixtures[i], &cfgs[i], &desc[i], &ch);
        if (st != BZ_OK) {
            delete b;
            return st;
        }
        b->ch_smem = b->ch_smem && ch;
    }
    // staging policy: every mixture's channel choice from its cumulative table in global memory
    if (opts && opts->channels_in_l2) b->ch_smem = false;
    b->smem = 0;
    for (int i = 0; i < n; ++i) {
        desc[i].stage_bytes = b->ch_smem ? desc[i].lay.stage_all : desc[i].lay.stage_tables;
        b->smem = std::max(b->smem, (size_t)desc[i].stage_bytes);
    }
    int bps = bz::batch_occupancy(precision, b->ch_smem, b->ext, b->wide, b->bfield, b->block, b->smem);
    if (bps < 1) {
        delete b;
        return fail(BZ_ECUDA, "batch kernel cannot be resident with these tables");
    }
    if (opts && opts->blocks_per_sm > 0 && opts->blocks_per_sm < bps) bps = opts->blocks_per_sm;
    uint64_t total = 0;
    for (int i = 0; i < n; ++i) total += cfgs[i].n_electrons;
    const uint32_t tile = (opts && opts->tile_particles > 0) ? (uint32_t)opts->tile_particles
                                                             : tile_size_for(total, (uint64_t)ctx->sm_count * bps, 16);
    // tiles, grouped by mixture (tables), then by swarm
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return desc[x].blob < desc[y].blob; });
    std::vector<std::pair<uint32_t, uint64_t>> work;
    for (int i : order) work.emplace_back((uint32_t)i, cfgs[i].n_electrons);
    std::vector<uint4> tiles;
    const uint32_t min_tile = std::min<uint32_t>((uint32_t)(b->block + 255) / 256 * 256, tile);
    guided_tiles(work, tile, (uint64_t)ctx->sm_count * bps, min_tile, &tiles);
    b->n_tiles = (int)tiles.size();
    b->grid = std::min(ctx->sm_count * bps, b->n_tiles);
    // one device allocation for everything
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    const size_t o_desc = take(sizeof(bz::RunArgs) * n), o_tiles = take(sizeof(uint4) * tiles.size());
    const size_t o_ctr = take(sizeof(unsigned int) * (2 + n));
    const size_t o_targs = take(sizeof(bz::TallyArgs) * n), o_tal = take(sizeof(bz_tallies) * n);
    std::vector<size_t> o_part(n), o_p1(n), o_p2(n), o_gs(n);
    std::vector<int> tb(n);
    b->n_el.resize(n);
    b->id_offset.resize(n);
    for (int i = 0; i < n; ++i) b->id_offset[i] = cfgs[i].id_offset;
    b->max_tblocks = 1;
    for (int i = 0; i < n; ++i) {
        const uint64_t m = cfgs[i].n_electrons;
        b->n_el[i] = m;
        o_part[i] = take((6 * 8 + 4 * 4 + 7 * 4) * m + 17 * 256);
        tb[i] = bz::tally_blocks(m, ctx->sm_count);
        b->max_tblocks = std::max(b->max_tblocks, tb[i]);
        o_p1[i] = take(sizeof(double) * tb[i] * bz::kGroups * bz::kQ1);
        o_p2[i] = take(sizeof(double) * tb[i] * bz::kGroups * bz::kQ2);
        o_gs[i] = take(sizeof(double) * (bz::kGroups * (bz::kQ1 + bz::kQ2) + 8));
    }
    b->bytes = off;
    // the set-up copies, from pinned staging; the library's own pool allocates
    // in their stream's order
    PinnedStage stage(ctx, sizeof(bz::RunArgs) * n + sizeof(uint4) * tiles.size() + sizeof(bz::TallyArgs) * n + 48);
    SyncCopies up;
    b->mem = (uint8_t *)dev_alloc(ctx, b->bytes, ctx->custom_alloc ? (cudaStream_t)0 : up.s);
    if (!b->mem) {
        delete b;
        return fail(BZ_ENOMEM, "device allocation of the batch");
    }
    ctx_retain(ctx);
    uint8_t *M = b->mem;
    b->desc = (bz::RunArgs *)(M + o_desc);
    b->tiles = (uint4 *)(M + o_tiles);
    b->tile_counter = (unsigned int *)(M + o_ctr);
    b->errs = b->tile_counter + 2;
    b->targs = (bz::TallyArgs *)(M + o_targs);
    b->tallies_dev = (bz_tallies *)(M + o_tal);
    std::vector<bz::TallyArgs> targs(n);
    b->p.resize(n);
    for (int i = 0; i < n; ++i) {
        const uint64_t m = b->n_el[i];
        size_t q = o_part[i];
        auto sub = [&](size_t bytes) { size_t o = q; q = align256(q + bytes); return (void *)(M + o); };
        bz::ParticlesDev &P = b->p[i];
        P.x = (double *)sub(8 * m); P.y = (double *)sub(8 * m); P.z = (double *)sub(8 * m); P.t = (double *)sub(8 * m);
        P.se = (double *)sub(8 * m); P.se2 = (double *)sub(8 * m);
        P.vx = (float *)sub(4 * m); P.vy = (float *)sub(4 * m); P.vz = (float *)sub(4 * m); P.nup = (float *)sub(4 * m);
        P.n_real = (uint32_t *)sub(4 * m); P.n_null = (uint32_t *)sub(4 * m); P.n_fail = (uint32_t *)sub(4 * m);
        P.n_ion = (uint32_t *)sub(4 * m); P.n_att = (uint32_t *)sub(4 * m); P.steps = (uint32_t *)sub(4 * m);
        P.status = (uint32_t *)sub(4 * m);
        desc[i].out = P;
        desc[i].err = b->errs + i;
        desc[i].counter = nullptr;
        bz::TallyArgs &t = targs[i];
        memset(&t, 0, sizeof t);
        t.x = P.x; t.y = P.y; t.z = P.z; t.t = P.t; t.se = P.se; t.se2 = P.se2;
        t.n_real = P.n_real; t.n_null = P.n_null; t.n_fail = P.n_fail; t.n_ion = P.n_ion; t.n_att = P.n_att;
        t.status = P.status; t.steps = P.steps;
        t.n = m;
        t.id_offset = cfgs[i].id_offset;
        t.part1 = (double *)(M + o_p1[i]);
        t.part2 = (double *)(M + o_p2[i]);
        t.gsum = (double *)(M + o_gs[i]);
        t.blocks = tb[i];
        t.E_V_m = cfgs[i].e_over_n_Td * bz::kTownsend * mixtures[i]->cm.n_total;
        t.n_total = mixtures[i]->cm.n_total;
        t.nu_trial = desc[i].nu0;
        t.err = b->errs + i;
        t.out = b->tallies_dev + i;
    }
    b->targs_host = targs;
    up.add(b->desc, stage.put(desc.data(), sizeof(bz::RunArgs) * n), sizeof(bz::RunArgs) * n, cudaMemcpyHostToDevice);
    up.add(b->tiles, stage.put(tiles.data(), sizeof(uint4) * tiles.size()), sizeof(uint4) * tiles.size(),
           cudaMemcpyHostToDevice);
    up.add(b->targs, stage.put(targs.data(), sizeof(bz::TallyArgs) * n), sizeof(bz::TallyArgs) * n,
           cudaMemcpyHostToDevice);
    e = up.wait();
    if (e == cudaSuccess) {
        b->tallies_host = (bz_tallies *)pinned_block(ctx, sizeof(bz_tallies) * n, &b->tallies_cap);
        if (!b->tallies_host) e = cudaErrorMemoryAllocation;
    }
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaEventCreate(&b->ev[i]);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    if (e == cudaSuccess && b->use_graph) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        bz_destroy_batch(b);
        return cuda_fail(e, "batch set-up");
    }
    if (b->use_graph) {
        // make sure the kernels' shared-memory limits are set before capture
        bz::batch_occupancy(precision, b->ch_smem, b->ext, b->wide, b->bfield, b->block, b->smem);
        for (int part = 0; part < 2 && e == cudaSuccess; ++part) {
            e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
            cudaError_t e1 = (e == cudaSuccess) ? batch_part(b, part, b->cap) : e;
            cudaError_t e2 = cudaStreamEndCapture(b->cap, &b->graph[part]);
            if (e == cudaSuccess) e = (e1 != cudaSuccess) ? e1 : e2;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec[part], b->graph[part], 0);
        }
        if (e != cudaSuccess) {
            bz_destroy_batch(b);
            return cuda_fail(e, "batch graph capture");
        }
    }
    *out = b;
    return BZ_OK;
}

bz_status bz_launch_batch(bz_batch *b, void *stream)
{
    if (!b) return fail(BZ_EINVAL, "null batch");
    cudaError_t e = cudaSetDevice(b->ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (e == cudaSuccess && b->launched) e = cudaEventSynchronize(b->done);
    if (e != cudaSuccess) return cuda_fail(e, "batch launch");
    bz_status st = batch_sequence(b, s);
    if (st != BZ_OK) return st;
    e = cudaEventRecord(b->done, s);
    if (e != cudaSuccess) return cuda_fail(e, "batch launch");
    b->launched = true;
    return BZ_OK;
}

bz_status bz_batch_read_tallies(bz_batch *b, bz_tallies *out)
{
    if (!b || !out) return fail(BZ_EINVAL, "null argument");
    if (!b->launched) return fail(BZ_EINVAL, "batch not launched");
    cudaError_t e = cudaEventSynchronize(b->done);
    if (e != cudaSuccess) return cuda_fail(e, "batch");
    bz_status st = BZ_OK;
    for (int i = 0; i < b->n; ++i) {
        out[i] = b->tallies_host[i];
        if (out[i].error_flags & BZ_ERR_STAGE_TIMEOUT) st = fail(BZ_ETIMEOUT, "table staging timed out");
        else if ((out[i].error_flags & BZ_ERR_TRIAL) && st == BZ_OK) st = fail(BZ_ETRIAL, "trial frequency exceeded (fixed mode, or a binned retry that failed again)");
    }
    return st;
}

bz_status bz_batch_read_particles(bz_batch *b, int32_t i, const bz_particles *o)
{
    if (!b || !o || i < 0 || i >= b->n) return fail(BZ_EINVAL, "bad argument");
    cudaError_t e = b->launched ? cudaEventSynchronize(b->done) : cudaSuccess;
    if (e != cudaSuccess) return cuda_fail(e, "batch");
    const size_t m = b->n_el[i];
    const bz::ParticlesDev &p = b->p[i];
    struct { void *dst; const void *src; size_t bytes; } cp[] = {
        {o->x, p.x, 8 * m}, {o->y, p.y, 8 * m}, {o->z, p.z, 8 * m}, {o->t, p.t, 8 * m}, {o->sum_e, p.se, 8 * m},
        {o->sum_e2, p.se2, 8 * m}, {o->vx, p.vx, 4 * m}, {o->vy, p.vy, 4 * m}, {o->vz, p.vz, 4 * m},
        {o->nu_p, p.nup, 4 * m}, {o->n_real, p.n_real, 4 * m}, {o->n_null, p.n_null, 4 * m},
        {o->n_fail, p.n_fail, 4 * m}, {o->n_ion, p.n_ion, 4 * m}, {o->n_att, p.n_att, 4 * m},
        {o->steps, p.steps, 4 * m}, {o->status, p.status, 4 * m}};
    {
        SyncCopies rd;
        for (auto &c : cp)
            if (c.dst) rd.add(c.dst, c.src, c.bytes, cudaMemcpyDeviceToHost);
        if ((e = rd.wait()) != cudaSuccess) return cuda_fail(e, "copy of particle state");
    }
    for (uint64_t k = 0; k < m; ++k) {
        if (o->id) o->id[k] = b->id_offset[i] + k;
        if (o->t_birth) o->t_birth[k] = 0.0;
    }
    return BZ_OK;
}

bz_status bz_batch_timing(bz_batch *b, double *step_ms, double *tally_ms)
{
    if (!b || !b->launched) return fail(BZ_EINVAL, "batch not launched");
    cudaError_t e = cudaEventSynchronize(b->done);
    float a = 0.f, c = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&a, b->ev[0], b->ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&c, b->ev[1], b->ev[2]);
    if (e != cudaSuccess) return cuda_fail(e, "batch timing");
    if (step_ms) *step_ms = a;
    if (tally_ms) *tally_ms = c;
    return BZ_OK;
}

void bz_destroy_batch(bz_batch *b)
{
    if (!b) return;
    cudaSetDevice(b->ctx->device);
    if (b->launched) cudaEventSynchronize(b->done);
    for (int i = 0; i < 2; ++i) {
        if (b->exec[i]) cudaGraphExecDestroy(b->exec[i]);
        if (b->graph[i]) cudaGraphDestroy(b->graph[i]);
    }
    if (b->cap) cudaStreamDestroy(b->cap);
    for (int i = 0; i < 3; ++i)
        if (b->ev[i]) cudaEventDestroy(b->ev[i]);
    if (b->done) cudaEventDestroy(b->done);
    bz_ctx *ctx = b->ctx;
    pinned_block_release(ctx, b->tallies_host, b->tallies_cap);
    if (b->mem) {
        // the batch's work is complete (waited above), so the memory is free on any stream
        dev_free(ctx, b->mem, b->bytes, 0);
        ctx_release(ctx);
    }
    delete b;
}

bz_status bz_batch_query(bz_batch *b)
{
    if (!b || !b->launched) return fail(BZ_EINVAL, "batch not launched");
    cudaError_t e = cudaEventQuery(b->done);
    if (e == cudaErrorNotReady) return BZ_ENOTREADY;
    if (e != cudaSuccess) return cuda_fail(e, "batch");
    return BZ_OK;
}

// ---------------------------------------------------------------------------
// Group sums: merging one swarm run in parts (id ranges on several ranks or
// launches) into one set of tallies
// ---------------------------------------------------------------------------
static bz_status group_sums1_of(const bz::TallyArgs &t, cudaEvent_t done, double *out)
{
    if (!out) return fail(BZ_EINVAL, "null output");
    cudaError_t e = cudaEventSynchronize(done);
    std::vector<double> g((size_t)bz::kGroups * bz::kGS);
    if (e == cudaSuccess) {
        SyncCopies rd;
        rd.add(g.data(), t.gsum, sizeof(double) * g.size(), cudaMemcpyDeviceToHost);
        e = rd.wait();
    }
    if (e != cudaSuccess) return cuda_fail(e, "group sums");
    for (int k = 0; k < bz::kGroups; ++k)
        for (int q = 0; q < bz::kQ1; ++q) out[k * bz::kQ1 + q] = g[(size_t)k * bz::kGS + q];
    return BZ_OK;
}

static bz_status group_sums2_of(const bz::TallyArgs &t, cudaEvent_t done, cudaStream_t s, const double *drift,
                                double *out)
{
    if (!drift || !out) return fail(BZ_EINVAL, "null argument");
    cudaError_t e = cudaEventSynchronize(done);
    if (e == cudaSuccess) e = bz::launch_group_sums2(t, drift, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    std::vector<double> g((size_t)bz::kGroups * bz::kGS);
    if (e == cudaSuccess) {
        SyncCopies rd;
        rd.add(g.data(), t.gsum, sizeof(double) * g.size(), cudaMemcpyDeviceToHost);
        e = rd.wait();
    }
    if (e != cudaSuccess) return cuda_fail(e, "group sums about the given drift");
    for (int k = 0; k < bz::kGroups; ++k)
        for (int q = 0; q < bz::kQ2; ++q) out[k * bz::kQ2 + q] = g[(size_t)k * bz::kGS + bz::kQ1 + q];
    return BZ_OK;
}

bz_status bz_swarm_group_sums1(bz_swarm *sw, double *out)
{
    if (!sw) return fail(BZ_EINVAL, "null swarm");
    cudaSetDevice(sw->ctx->device);
    return group_sums1_of(sw->targs, sw->done, out);
}

bz_status bz_swarm_group_sums2(bz_swarm *sw, const double *drift, double *out)
{
    if (!sw) return fail(BZ_EINVAL, "null swarm");
    cudaSetDevice(sw->ctx->device);
    return group_sums2_of(sw->targs, sw->done, sw->stream, drift, out);
}

bz_status bz_batch_group_sums1(bz_batch *b, int32_t i, double *out)
{
    if (!b || i < 0 || i >= b->n || !b->launched) return fail(BZ_EINVAL, "bad batch, swarm index, or not launched");
    cudaSetDevice(b->ctx->device);
    return group_sums1_of(b->targs_host[i], b->done, out);
}

bz_status bz_batch_group_sums2(bz_batch *b, int32_t i, const double *drift, double *out)
{
    if (!b || i < 0 || i >= b->n || !b->launched) return fail(BZ_EINVAL, "bad batch, swarm index, or not launched");
    cudaSetDevice(b->ctx->device);
    return group_sums2_of(b->targs_host[i], b->done, (cudaStream_t)0, drift, out);
}

bz_status bz_drift_from_group_sums(const double *g1, double *drift)
{
    if (!g1 || !drift) return fail(BZ_EINVAL, "null argument");
    std::vector<double> g((size_t)bz::kGroups * bz::kGS, 0.0);
    for (int k = 0; k < bz::kGroups; ++k)
        for (int q = 0; q < bz::kQ1; ++q) g[(size_t)k * bz::kGS + q] = g1[k * bz::kQ1 + q];
    bz::drift_of_groups(g.data(), drift);
    return BZ_OK;
}

bz_status bz_finalize_group_sums(const double *g1, const double *g2, const bz_merge_info *info, bz_tallies *out)
{
    if (!g1 || !g2 || !info || !out) return fail(BZ_EINVAL, "null argument");
    std::vector<double> g((size_t)bz::kGroups * bz::kGS + 8, 0.0);
    for (int k = 0; k < bz::kGroups; ++k) {
        for (int q = 0; q < bz::kQ1; ++q) g[(size_t)k * bz::kGS + q] = g1[k * bz::kQ1 + q];
        for (int q = 0; q < bz::kQ2; ++q) g[(size_t)k * bz::kGS + bz::kQ1 + q] = g2[k * bz::kQ2 + q];
    }
    double *S = g.data() + (size_t)bz::kGroups * bz::kGS;
    bz::drift_of_groups(g.data(), S);
    bz::GroupScalars X;
    X.E_V_m = info->e_over_n_Td * bz::kTownsend * info->n_total_m3;
    X.n_total = info->n_total_m3;
    X.nu_trial = info->nu_trial;
    X.n_spawned = info->n_spawned;
    X.n_capped = info->n_capped;
    X.error_flags = info->error_flags;
    bz::tallies_of_groups(g.data(), S, X, out);
    return BZ_OK;
}

bz_status bz_step_replay(bz_ctx *ctx, const bz_mixture *mix, const bz_swarm_config *cfg, int64_t n,
                         const double *state_in_dev, const uint64_t *ids_dev, const uint32_t *steps_dev,
                         double *state_out_dev, int32_t *decision_dev, double *eps_dev, void *stream)
{
    if (!ctx || !mix || !cfg) return fail(BZ_EINVAL, "null argument");
    if (n < 0) return fail(BZ_EINVAL, "n must be >= 0");
    if (n == 0) return BZ_OK;
    if (!state_in_dev || !ids_dev || !steps_dev || !state_out_dev || !decision_dev || !eps_dev)
        return fail(BZ_EINVAL, "null buffer");
    bz_status vs = validate_config(cfg);
    if (vs != BZ_OK) return vs;
    if (adaptive(cfg)) return fail(BZ_EINVAL, "single steps replay the lazy, fixed or windowed trial frequency");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    bz::ReplayArgs r;
    bool ch_smem;
    bz_status st = prepare_run(mix, cfg, &r.run, &ch_smem);
    if (st != BZ_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *err = (uint32_t *)dev_alloc(ctx, 256, s);
    if (!err) return fail(BZ_ENOMEM, "device allocation");
    cudaMemsetAsync(err, 0, 4, s);
    r.run.err = err;
    r.n = n;
    r.state_in = state_in_dev;
    r.ids = ids_dev;
    r.steps = steps_dev;
    r.state_out = state_out_dev;
    r.decision = decision_dev;
    r.eps_io = eps_dev;
    const int block = 256;
    int64_t g = (n + block - 1) / block;
    const int grid = (int)(g < ctx->sm_count * 4 ? g : ctx->sm_count * 4);
    e = bz::launch_replay(cfg->precision, ch_smem, r, grid, block, s);
    dev_free(ctx, err, 256, s);
    if (e != cudaSuccess) return cuda_fail(e, "replay launch");
    return BZ_OK;
}

bz_status bz_philox(bz_ctx *ctx, int64_t n, const uint32_t *ctr_dev, uint64_t key, uint32_t *out_dev, void *stream)
{
    if (!ctx) return fail(BZ_EINVAL, "null context");
    if (n < 0) return fail(BZ_EINVAL, "n must be >= 0");
    if (n > 0 && (!ctr_dev || !out_dev)) return fail(BZ_EINVAL, "null buffer");
    if (((uintptr_t)ctr_dev | (uintptr_t)out_dev) & 15) return fail(BZ_EINVAL, "buffers must be 16-byte aligned");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = bz::launch_philox(n, ctr_dev, key, out_dev, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "philox launch");
    return BZ_OK;
}

}  // extern "C"
