// noalloc.cu -- bz_reduce_tallies_noalloc: the FP64 swarm-tally reduction
// with its scratch in a static device array instead of allocated memory.
//
// Who needs it: callers that cannot allocate device memory where they want
// swarm statistics -- a process whose device memory is held entirely by
// another allocator (a framework's caching pool, a serving process with a
// fixed HBM plan), where cudaMalloc fails or fragments the pool, and
// latency-sensitive loops in which cudaMalloc / cudaFree would synchronize
// the device.  The reduction itself is the same four kernels that
// bz_run_swarm launches (two FP64 passes over the particles plus two small
// fixed-order reductions); only where their scratch lives differs.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>
#include <string>

#include "bz.h"
#include "kernels.h"

namespace {

// Scratch of the reduction: per-block partial sums of both passes, the group
// sums with the drift summary, and one error word.  Every GPU that loads
// libbz.so holds it until the process exits.
constexpr size_t kPart1 = (size_t)BZ_NOALLOC_MAX_BLOCKS * bz::kGroups * bz::kQ1;
constexpr size_t kPart2 = (size_t)BZ_NOALLOC_MAX_BLOCKS * bz::kGroups * bz::kQ2;
constexpr size_t kGsum = (size_t)bz::kGroups * (bz::kQ1 + bz::kQ2) + 8;
static_assert(bz::kQ1 + bz::kQ2 == 29, "scratch size formula in bz.h assumes 29 quantities");
static_assert(8 * (kPart1 + kPart2 + kGsum) + 256 <= BZ_NOALLOC_SCRATCH_BYTES, "scratch too small");

static __device__ __align__(256) unsigned char g_scratch[BZ_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices];  // device address of g_scratch, per device

bz_status fail(bz_status s, const std::string &msg)
{
    bz::set_last_error(msg);
    return s;
}

// Set-up, once per device, with that device current.
bz_status scratch_address(int device, unsigned char **out)
{
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return fail(BZ_ECUDA, std::string("cudaGetSymbolAddress of the scratch array: ") + cudaGetErrorString(e));
        g_scratch_ptr[device] = p;
    }
    *out = (unsigned char *)g_scratch_ptr[device];
    return BZ_OK;
}

}  // namespace

extern "C" bz_status bz_reduce_tallies_noalloc(const bz_particle_arrays *in, uint64_t n, uint64_t id_offset,
                                               double e_over_n_Td, double n_total_m3, double nu_trial,
                                               bz_tallies *out_dev, void *stream)
{
    if (!in || !out_dev) return fail(BZ_EINVAL, "null argument");
    if (n == 0) return fail(BZ_EINVAL, "n must be >= 1");
    if (n > (uint64_t)BZ_NOALLOC_MAX_PARTICLES)
        return fail(BZ_EBUDGET, "n exceeds BZ_NOALLOC_MAX_PARTICLES (16777216) of the allocation-free reduction");
    if (!in->x || !in->y || !in->z || !in->t || !in->sum_e || !in->sum_e2 || !in->n_real || !in->n_null ||
        !in->n_fail || !in->n_ion || !in->n_att || !in->status)
        return fail(BZ_EINVAL, "null particle array");
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return fail(BZ_ECUDA, cudaGetErrorString(e));
    if (device < 0 || device >= kMaxDevices) return fail(BZ_EINVAL, "device index out of range");
    unsigned char *S;
    bz_status st = scratch_address(device, &S);
    if (st != BZ_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    bz::TallyArgs t;
    memset(&t, 0, sizeof t);
    t.x = in->x; t.y = in->y; t.z = in->z; t.t = in->t; t.se = in->sum_e; t.se2 = in->sum_e2;
    t.n_real = in->n_real; t.n_null = in->n_null; t.n_fail = in->n_fail; t.n_ion = in->n_ion;
    t.n_att = in->n_att; t.status = in->status;
    t.steps = in->steps;
    t.n = n;
    t.id_offset = id_offset;
    t.blocks = (int)((n + BZ_NOALLOC_SPAN - 1) / BZ_NOALLOC_SPAN);
    t.part1 = (double *)S;
    t.part2 = t.part1 + kPart1;
    t.gsum = t.part2 + kPart2;
    uint32_t *err = (uint32_t *)(t.gsum + kGsum);  // error word: must read 0, the rest is overwritten
    t.err = err;
    t.E_V_m = e_over_n_Td * bz::kTownsend * n_total_m3;
    t.n_total = n_total_m3;
    t.nu_trial = nu_trial;
    t.out = out_dev;
    e = cudaMemsetAsync(err, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess) e = bz::launch_tallies(t, s);
    if (e != cudaSuccess) return fail(BZ_ECUDA, cudaGetErrorString(e));
    return BZ_OK;
}
