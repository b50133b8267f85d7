// Launch accounting and optional per-kernel CUDA-event timing.
//
// Every kernel launch of the library goes through LDNI_LAUNCH, which counts
// it and, when a caller has installed event slots with ldni_profile_set and
// the kernel id passes the filter, records a begin event before and an end
// event after the launch on the same stream.
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

namespace ldni {

enum KernelId : int {
    K_NONE = 0,
    K_COUNT_TRI = 1,
    K_COUNT_BIG = 2,
    K_SCAN_CHUNK = 3,
    K_SCAN_TOP = 4,
    K_SCAN_DOWN = 5,
    K_FILL_TRI = 6,
    K_FILL_BIG = 7,
    K_SORT = 8,
    K_BOOL_COUNT = 9,
    K_BOOL_WRITE = 10,
    K_VOL_PARTIAL = 11,
    K_VOL_FINAL = 12,
    K_BOOL_FUSED = 13,
    K_FEATURES = 14,
    K_CAPACITY = 15,
    K_LAYOUT = 16,
    K_ONEPASS = 17,
    K_ONEPASS_BIG = 18,
    K_REDO = 19,
    K_GATHER = 20,
    K_MLP = 21,
    K_GRAD = 22,
    K_BATCH = 23,
    K_NODES = 24,
    K_ORDER = 25,
    K_OFFSET = 26,
    K_CODEC = 27,
    K_CONTOUR = 28,
    K_CHAIN = 29,
    K_BIN = 30,
    K_TILE = 31,
    K_RETIRED_32 = 32,  // the tile scan of the former three-launch Boolean
    K_NUM = 33
};

struct ProfState {
    cudaEvent_t *begin = nullptr;
    cudaEvent_t *end = nullptr;
    int32_t *ids = nullptr;
    int32_t cap = 0;
    int32_t next = 0;
    int32_t filter = 0;  // 0 = every kernel, else one KernelId
};

ProfState &prof_state();
std::atomic<uint64_t> &launch_counter();

// Inside a stream capture the record becomes a graph node that fires on
// every replay (external record); outside one it is an ordinary record.
inline unsigned record_flags(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) cs = cudaStreamCaptureStatusNone;
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
}

inline int prof_begin(int id, cudaStream_t s) {
    launch_counter().fetch_add(1, std::memory_order_relaxed);
    ProfState &P = prof_state();
    if (P.cap <= 0 || (P.filter != 0 && P.filter != id)) return -1;
    const int slot = P.next % P.cap;
    if (!P.begin[slot] || !P.end[slot]) return -1;
    P.next++;
    if (P.ids) P.ids[slot] = id;
    cudaEventRecordWithFlags(P.begin[slot], s, record_flags(s));
    return slot;
}

inline void prof_end(int slot, cudaStream_t s) {
    if (slot < 0) return;
    cudaEventRecordWithFlags(prof_state().end[slot], s, record_flags(s));
}

}  // namespace ldni

#define LDNI_LAUNCH(id, stream, ...)                  \
    do {                                              \
        const int ldni_slot_ = ::ldni::prof_begin((id), (stream)); \
        __VA_ARGS__;                                  \
        ::ldni::prof_end(ldni_slot_, (stream));       \
    } while (0)
