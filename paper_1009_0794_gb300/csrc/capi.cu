// Small C-ABI helpers: error strings, version, grid from a bounding box.
#include <atomic>
#include <cmath>
#include <mutex>

#include "ldni_host.h"
#include "lookback.cuh"

extern "C" const char *ldni_strerror(int code) {
    switch (code) {
        case LDNI_OK: return "ok";
        case LDNI_EINVAL: return "invalid argument";
        case LDNI_EGRID_MISMATCH: return "Boolean operands are sampled on different grids";
        case LDNI_EODD: return "an input ray has an odd number of samples";
        case LDNI_ETOOLARGE: return "size beyond the int32 CSR range";
        case LDNI_EWORKSPACE: return "workspace smaller than the size query";
        case LDNI_ECUDA: return "CUDA runtime error";
        case LDNI_ETIMEOUT: return "bounded device wait expired";
        case LDNI_ERANGE: return "vertex outside the snappable range of the grid";
        case LDNI_ECAPACITY: return "output capacity smaller than the sample count";
        default: return "unknown ldni error";
    }
}

namespace ldni {
namespace {
thread_local cudaError_t g_last_cuda_error = cudaSuccess;
}
int cuda_fail(cudaError_t e) {
    g_last_cuda_error = e;
    return LDNI_ECUDA;
}
}  // namespace ldni

extern "C" const char *ldni_last_cuda_error(void) {
    return ldni::g_last_cuda_error == cudaSuccess ? "no CUDA error" : cudaGetErrorString(ldni::g_last_cuda_error);
}

extern "C" int ldni_version(void) { return 100; }

extern "C" int ldni_grid_from_bbox(const float *bbox, int32_t res, ldni_grid_t *grid) {
    if (!bbox || !grid || res < 1 || res > 8192) return LDNI_EINVAL;
    float w = 0.0f;
    for (int k = 0; k < 3; ++k) {
        if (!std::isfinite(bbox[k]) || !std::isfinite(bbox[k + 3]) || bbox[k + 3] < bbox[k]) return LDNI_EINVAL;
        const float e = bbox[k + 3] - bbox[k];
        if (e > w) w = e;
    }
    if (!(w > 0.0f)) return LDNI_EINVAL;
    for (int k = 0; k < 3; ++k) grid->origin[k] = bbox[k];
    grid->width = w;
    grid->res = res;
    return LDNI_OK;
}

// ---- launch accounting and optional per-kernel event timing -------------

namespace ldni {
ProfState &prof_state() {
    static ProfState s;
    return s;
}
std::atomic<uint64_t> &launch_counter() {
    static std::atomic<uint64_t> c{0};
    return c;
}
}  // namespace ldni

extern "C" int ldni_profile_set(void **begin_events, void **end_events, int32_t *kernel_ids, int32_t capacity,
                                int32_t filter) {
    ldni::ProfState &P = ldni::prof_state();
    if (capacity < 0 || filter < 0 || filter >= ldni::K_NUM) return LDNI_EINVAL;
    if (capacity > 0 && (!begin_events || !end_events)) return LDNI_EINVAL;
    P.begin = reinterpret_cast<cudaEvent_t *>(begin_events);
    P.end = reinterpret_cast<cudaEvent_t *>(end_events);
    P.ids = kernel_ids;
    P.cap = capacity;
    P.next = 0;
    P.filter = filter;
    return LDNI_OK;
}

extern "C" int64_t ldni_profile_recorded(void) { return ldni::prof_state().next; }

extern "C" uint64_t ldni_launch_count(void) { return ldni::launch_counter().load(); }

extern "C" const char *ldni_kernel_name(int32_t id) {
    static const char *names[ldni::K_NUM] = {"none",       "count_tri",  "count_big", "unused",
                                             "scan_tiles", "scan",       "fill_tri",  "fill_big",
                                             "sort_rays",  "bool_count", "bool_write", "volume",
                                             "unused",     "boolean",    "features",  "capacity",
                                             "layout",     "onepass",    "onepass_big", "redo",
                                             "gather",     "mlp",        "adjoint",   "batch",      "nodes",     "order",     "offset",    "normals8",  "contour",   "chain",     "bin",       "tile",      "unused"};
    return (id >= 0 && id < ldni::K_NUM) ? names[id] : "unknown";
}

// ---- bounded device waits ------------------------------------------------------
namespace ldni {
namespace {
std::atomic<int> g_wait_limit{kDefaultWaitPolls};

// One warp polls, with the library's bounded wait, a shared word that nothing
// sets; after `polls` polls it gives up and records LDNI_ST_TIMEOUT.
__global__ void wait_selftest_kernel(ldni_info_t *info, int polls) {
    __shared__ unsigned long long never_set;
    if (threadIdx.x == 0) never_set = 0;
    __syncwarp();
    int spins = 0;
    bool timed_out = false;
    while (true) {
        const bool missing = (*reinterpret_cast<volatile unsigned long long *>(&never_set) & ~kValueMask) == 0;
        if (!__any_sync(0xffffffffu, missing)) break;
        if (++spins > polls) {
            timed_out = true;
            break;
        }
        __nanosleep(32);
    }
    if (timed_out && threadIdx.x == 0) atomicOr(&info->status, LDNI_ST_TIMEOUT);
}
}  // namespace

int wait_limit() { return g_wait_limit.load(); }
}  // namespace ldni

extern "C" int ldni_set_wait_limit(int32_t polls) {
    if (polls < 0) return LDNI_EINVAL;
    ldni::g_wait_limit.store(polls == 0 ? ldni::kDefaultWaitPolls : polls);
    return LDNI_OK;
}

extern "C" int32_t ldni_get_wait_limit(void) { return ldni::g_wait_limit.load(); }

extern "C" int32_t ldni_build_checked(void) { return ldni::kChecked ? 1 : 0; }

extern "C" int ldni_wait_selftest(ldni_info_t *info, void *stream) {
    if (!info) return LDNI_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    LDNI_LAUNCH(ldni::K_NONE, s, ldni::wait_selftest_kernel<<<1, 32, 0, s>>>(info, ldni::wait_limit()));
    return ldni::cuda_status();
}

// ---- launch tuning -----------------------------------------------------------
namespace ldni {
namespace {
constexpr ldni_tuning_t kDefaultTuning = {512, 4096, 16, -1};
std::mutex g_tuning_mu;
ldni_tuning_t g_tuning = kDefaultTuning;

bool tuning_ok(const ldni_tuning_t &t) {
    const int r = t.bool_tile_rays;
    return (r == 256 || r == 512 || r == 1024 || r == 2048) && t.bool_stage_samples >= 0 &&
           t.bool_stage_samples <= 16384 && t.tri_blocks_per_sm >= 1 && t.tri_blocks_per_sm <= 64 &&
           t.bool_split >= -1 && t.bool_split <= 1;
}
}  // namespace

ldni_tuning_t current_tuning() {
    std::lock_guard<std::mutex> lock(g_tuning_mu);
    return g_tuning;
}
}  // namespace ldni

extern "C" int ldni_get_tuning(ldni_tuning_t *t) {
    if (!t) return LDNI_EINVAL;
    *t = ldni::current_tuning();
    return LDNI_OK;
}

extern "C" int ldni_set_tuning(const ldni_tuning_t *t) {
    const ldni_tuning_t v = t ? *t : ldni::kDefaultTuning;
    if (!ldni::tuning_ok(v)) return LDNI_EINVAL;
    std::lock_guard<std::mutex> lock(ldni::g_tuning_mu);
    ldni::g_tuning = v;
    return LDNI_OK;
}
