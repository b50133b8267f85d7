// The per-ray merge of two sorted sample lists by inside-counters (Section
// 4.1), shared by the Boolean (boolean.cu) and the union chain (chain.cu).
//
// Walking the distinct depths of both lists in order, every sample toggles
// its solid's state (odd-to-even ranges are inside, Section 2); equal depths
// of A and B are one event; the output state op(inA, inB) changes exactly at
// the result's boundary samples.  An entering sample waits until its exit is
// known, so an interval thinner than eps (Section 4.1.1) is dropped without a
// second pass.
#pragma once

#include "ldni.h"

namespace ldni {

// Truth table of an operation: bit (2 inA + inB) = op(inA, inB).
__device__ __forceinline__ unsigned op_table(int op) {
    return op == LDNI_OP_UNION ? 0xEu : (op == LDNI_OP_INTER ? 0x8u : 0x4u);
}

// The merge of one ray over index ranges [a, ae) of dA and [b, be) of dB.
// Every sample is read once.  emit(pend_from_b, pend_idx, cur_from_b,
// cur_idx, m) is called for every kept interval (entering sample, leaving
// sample) with m = samples so far.  A depth that equals nothing, itself
// included (NaN, outside the method's inputs), is consumed on its own so the
// walk always ends.
template <class Idx, class PA, class PB, class EmitF>
__device__ __forceinline__ int merge_core(PA dA, Idx a, Idx ae, PB dB, Idx b, Idx be, int op, float eps,
                                          EmitF emit) {
    const unsigned table = op_table(op);
    unsigned state = 0;  // bit 1: inside A, bit 0: inside B
    bool out = false;
    bool pend_b = false;
    Idx pend_i = 0;
    float pend_d = 0.0f;
    int m = 0;
    float da = a < ae ? dA[a] : 0.0f;
    float db = b < be ? dB[b] : 0.0f;
    while (a < ae || b < be) {
        const bool takeA = a < ae && (b >= be || !(db < da));
        const float d = takeA ? da : db;
        const Idx fa = a, fb = b;
        while (a < ae && da == d) {
            ++a;
            da = a < ae ? dA[a] : 0.0f;
        }
        while (b < be && db == d) {
            ++b;
            db = b < be ? dB[b] : 0.0f;
        }
        if (a == fa && b == fb) {  // NaN guard
            if (takeA) {
                ++a;
                da = a < ae ? dA[a] : 0.0f;
            } else {
                ++b;
                db = b < be ? dB[b] : 0.0f;
            }
        }
        const bool flipA = ((a - fa) & 1) != 0;
        state ^= (flipA ? 2u : 0u) | (((b - fb) & 1) ? 1u : 0u);
        const bool now = (table >> state) & 1u;
        if (now == out) continue;
        out = now;
        const bool cur_b = !flipA;
        const Idx cur_i = flipA ? fa : fb;
        if (now) {
            pend_b = cur_b;
            pend_i = cur_i;
            pend_d = d;
        } else if (!(__fsub_rn(d, pend_d) < eps)) {
            emit(pend_b, pend_i, cur_b, cur_i, m);
            m += 2;
        }
    }
    return m;
}

struct NoEmit {
    template <class Idx>
    __device__ __forceinline__ void operator()(bool, Idx, bool, Idx, int) const {}
};

}  // namespace ldni
