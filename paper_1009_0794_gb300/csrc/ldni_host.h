// Host-side helpers shared by the C-ABI entry points: workspace carving,
// grid validation and CUDA error mapping.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "ldni.h"
#include "ldni_device.cuh"
#include "prof.h"

namespace ldni {

constexpr size_t kAlign = 256;

inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Hands out aligned slices of one caller-provided workspace.  With base ==
// nullptr it only measures.
struct Carver {
    char *base;
    size_t off = 0;
    size_t cap;
    Carver(void *b, size_t c) : base(static_cast<char *>(b)), cap(c) {}
    template <class T>
    T *take(size_t count) {
        size_t at = align_up(off);
        off = at + count * sizeof(T);
        return base ? reinterpret_cast<T *>(base + at) : nullptr;
    }
    bool fits() const { return off <= cap; }
};

// Launch knobs (ldni_set_tuning), copied at launch time.
ldni_tuning_t current_tuning();

// Polls a bounded device wait makes before it gives up (ldni_set_wait_limit),
// passed to the kernels at launch time.
constexpr int kDefaultWaitPolls = 1 << 22;
int wait_limit();

inline bool grid_valid(const ldni_grid_t *g) {
    return g && g->res >= 1 && g->res <= 8192 && g->width > 0.0f && g->width < 3.0e38f;
}

// The sample arrays of a layer are present (capacity 0 needs none).
inline bool samples_ok(const ldni_layers_t &L) {
    return L.capacity == 0 || (L.depth && L.tri_id && (L.nrm8 || (L.nx && L.ny && L.nz)));
}

// Normal format of a layer: 1 packed 8-bit words, 0 FP32, -1 either (an
// empty layer may come without any sample array).
inline int layer_format(const ldni_layers_t &L) {
    if (L.nrm8) return 1;
    if (L.nx || L.capacity > 0) return 0;
    return -1;
}

// The operands and outputs of one call share a format: *packed receives it.
inline bool same_format(const ldni_layers_t *const *Ls, int n, bool *packed) {
    int f = -1;
    for (int k = 0; k < n; ++k) {
        const int g = layer_format(*Ls[k]);
        if (g < 0) continue;
        if (f >= 0 && g != f) return false;
        f = g;
    }
    *packed = f == 1;
    return true;
}

// Normal arrays as the kernels take them: FP32 in x, y, z, or the packed
// 8-bit words in x with y = z = nullptr.
inline void normal_arrays(const ldni_layers_t &L, float *&x, float *&y, float *&z) {
    if (L.nrm8) {
        x = reinterpret_cast<float *>(L.nrm8);
        y = z = nullptr;
    } else {
        x = L.nx;
        y = L.ny;
        z = L.nz;
    }
}

inline GridDev make_grid(const ldni_grid_t *g) {
    GridDev d;
    d.o[0] = g->origin[0];
    d.o[1] = g->origin[1];
    d.o[2] = g->origin[2];
    d.s = (float)((double)g->res * (double)kSubpix / (double)g->width);
    d.res = g->res;
    return d;
}

// Records e as the calling thread's last CUDA failure (ldni_last_cuda_error)
// and returns LDNI_ECUDA.
int cuda_fail(cudaError_t e);

// LDNI_ECUDA when a launch or an earlier asynchronous call failed, else LDNI_OK.
inline int cuda_status() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LDNI_OK : cuda_fail(e);
}

// cudaSuccess -> LDNI_OK, anything else recorded -> LDNI_ECUDA
inline int cuda_check(cudaError_t e) { return e == cudaSuccess ? LDNI_OK : cuda_fail(e); }

inline int num_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 152;
    }
    return sms;
}

// ---- CSR scan (scan.cu) ------------------------------------------------
// offsets[a][0..N] = exclusive prefix sum of counts[a][0..N-1], offsets[a][N]
// = total; info->n[info_base + a] = total; totals above 2^31-1 set
// LDNI_ST_TOOLARGE.  `partials` must hold csr_scan_partials(N) int64 per axis.
// With `tinfo`, tinfo[a][c] = (offset of count c * kScanChunk, sum of that
// chunk's counts) for every chunk c of kScanChunk counts.
// With `verify` (one-pass sampling), chunk c of image k whose tile has
// kcap[k][c] == 2 layers is also checked: every ray must have 0 crossings,
// or 2 of which exitc says exactly one leaves; otherwise over[k][c] and
// *any_over are set to 1 (the tile is redone exactly).
constexpr int kScanChunk = 4096;
struct ScanVerify {
    const int *exitc[3];
    const int *kcap[3];
    int *over[3];
    int *any_over;
};
size_t csr_scan_partials(long long N);
int csr_scan(const int *const *counts, int *const *offsets, int naxes, long long N, long long *partials,
             ldni_info_t *info, int info_base, cudaStream_t s, int2 *const *tinfo = nullptr,
             const ScanVerify *verify = nullptr);

}  // namespace ldni
