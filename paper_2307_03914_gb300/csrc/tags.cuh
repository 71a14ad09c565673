// tags.cuh -- tagged-slot reductions among the blocks of one launch (the
// on-chip MGS kernels, and the teams of the batched solver).
#pragma once

#include "common.cuh"
#include "tma.cuh"

namespace bspai {

__device__ __forceinline__ float tag_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double tag_add(double a, double b) { return __dadd_rn(a, b); }

// Tagged-slot reduction among G blocks (the grid of k_mgs_res, or a team).  Every block owns one slot per
// parity of the pass number; it publishes its partial sum there together with
// the reduction's sequence number, value and number travelling in the same
// 64-bit store (fp32: one word {seq, bits}; fp64: two words {seq, high half},
// {seq, low half}).  A block has the grid total once every slot carries the
// current number: no atomics, no fences and no separate read of the partials
// after a release.  The sequence numbers continue across launches (the count
// lives in GridBar::seq, advanced by block 0 after the kernel's last
// reduction), so slots left by earlier reductions never match.  The partials
// are added in the same fixed order as grid_wait (lane-strided, then a warp
// butterfly), so the total is the same in every block and in every run.
template <typename T>
struct TagWords;
template <>
struct TagWords<float> {
    static constexpr int W = 1;
};
template <>
struct TagWords<double> {
    static constexpr int W = 2;
};
constexpr int kTagMaxBlocks = 160;  // slots read per lane: kTagMaxBlocks / 32 (152 SMs)

__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void tag_publish(float v, unsigned long long* slot, unsigned seq) {
    st_relaxed_u64(slot, ((unsigned long long)seq << 32) | __float_as_uint(v));
}
__device__ __forceinline__ void tag_publish(double v, unsigned long long* slot, unsigned seq) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    st_relaxed_u64(slot, ((unsigned long long)seq << 32) | (b >> 32));
    st_relaxed_u64(slot + 1, ((unsigned long long)seq << 32) | (b & 0xffffffffull));
}
// true (and *v set) once the slot carries `seq`
__device__ __forceinline__ bool tag_read(const unsigned long long* slot, unsigned seq, float* v) {
    const unsigned long long a = ld_relaxed_u64(slot);
    if ((unsigned)(a >> 32) != seq) return false;
    *v = __uint_as_float((unsigned)a);
    return true;
}
__device__ __forceinline__ bool tag_read(const unsigned long long* slot, unsigned seq, double* v) {
    const unsigned long long a = ld_relaxed_u64(slot), b = ld_relaxed_u64(slot + 1);
    if ((unsigned)(a >> 32) != seq || (unsigned)(b >> 32) != seq) return false;
    *v = __longlong_as_double((long long)((a << 32) | (b & 0xffffffffull)));
    return true;
}

// tag_read on a copy of the slots in shared memory
__device__ __forceinline__ bool tag_read_smem(const unsigned long long* slot, unsigned seq, float* v) {
    const unsigned long long a = *slot;
    if ((unsigned)(a >> 32) != seq) return false;
    *v = __uint_as_float((unsigned)a);
    return true;
}
__device__ __forceinline__ bool tag_read_smem(const unsigned long long* slot, unsigned seq, double* v) {
    const unsigned long long a = slot[0], b = slot[1];
    if ((unsigned)(a >> 32) != seq || (unsigned)(b >> 32) != seq) return false;
    *v = __longlong_as_double((long long)((a << 32) | (b & 0xffffffffull)));
    return true;
}

template <typename T>
__device__ __forceinline__ void tag_arrive(T v, unsigned long long* tags, int set, unsigned seq, T* s_w,
                                           int G = -1) {
    if (G < 0) G = gridDim.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    if (lane == 0) s_w[w] = v;
    __syncthreads();
    if (w == 0) {
        T t = lane < nw ? s_w[lane] : T(0);
        t = warp_sum(t);
        if (lane == 0)
            tag_publish(t, tags + ((int64_t)set * G + blockIdx.x) * TagWords<T>::W, seq);
    }
}

// The lanes of one warp poll the G slots of `set` until all carry `seq`
// (giving up after tmo ns, or when another block has flagged an error) and
// add them in a fixed order (lane-strided, then a warp butterfly): every lane
// gets the total, the same in every block.  False after a timeout.
template <typename T>
__device__ __forceinline__ bool tag_poll_warp(const unsigned long long* tags, int set, unsigned seq, int G,
                                              GridBar* bar, unsigned long long tmo, T* total) {
    constexpr int MS = kTagMaxBlocks / 32;
    constexpr int TW = TagWords<T>::W;
    const int lane = threadIdx.x & 31;
    const unsigned long long* base = tags + (int64_t)set * G * TW;
    T val[MS];
    unsigned pending = 0;
#pragma unroll
    for (int m = 0; m < MS; ++m) {
        val[m] = T(0);
        if (lane + 32 * m < G) pending |= 1u << m;
    }
    bool ok = true;
    unsigned long long t0 = 0;
    for (int it = 0;; ++it) {
#pragma unroll
        for (int m = 0; m < MS; ++m)
            if ((pending >> m) & 1u)
                if (tag_read(base + (int64_t)(lane + 32 * m) * TW, seq, &val[m])) pending &= ~(1u << m);
        if (!__any_sync(0xffffffffu, pending != 0)) break;
        int stop = 0;
        if (lane == 0) {
            const unsigned long long now = globaltimer_ns();
            if (it == 0) t0 = now;
            if (now - t0 > tmo) {
                atomicExch(&bar->err, 1);
                stop = 1;
            } else if ((it & 63) == 63 && *(volatile int*)&bar->err) {
                stop = 1;
            }
        }
        if (__shfl_sync(0xffffffffu, stop, 0)) {
            ok = false;
            break;
        }
    }
    T t = T(0);
#pragma unroll
    for (int m = 0; m < MS; ++m)
        if (lane + 32 * m < G) t = tag_add(t, val[m]);
    *total = warp_sum(t);
    return ok;
}

// tag_poll_warp with the slots read by bulk copies (the TMA engine) into
// shared memory instead of by loads: each round lane 0 posts one copy of the
// G slots (16-byte aligned: from the even word at or below the set's first
// slot, a whole number of 16-byte units), the warp waits on the mbarrier and
// checks the tags.  In a kernel whose warps have just issued their loads of
// the next basis vector, those loads fill the SM's load path and an ordinary
// poll waits behind them; the copy engine's requests do not (measured on the
// MGS pass loop at 128 blocks x 16,384 rows: 2.06 against 2.89 us per pass).
// Same fixed order of the additions as tag_poll_warp, so the same total.
// s_slots: 2 kTagMaxBlocks + 2 words of shared memory (16-byte aligned);
// bar: an mbarrier initialised with count 1, used only by this warp; phase:
// the warp's count of completed copies on it (the same in every lane).
// False after a timeout (after waiting once more, bounded, for the copy in flight).
template <typename T>
__device__ __forceinline__ bool tag_poll_warp_bulk(const unsigned long long* tags, int set, unsigned seq, int G,
                                                   GridBar* bar, unsigned long long tmo, T* total,
                                                   unsigned long long* s_slots, uint64_t* mbar, unsigned& phase) {
    constexpr int MS = kTagMaxBlocks / 32;
    constexpr int TW = TagWords<T>::W;
    const int lane = threadIdx.x & 31;
    const int64_t first = (int64_t)set * G * TW;
    const int64_t a0 = first & ~(int64_t)1;
    const int skip = (int)(first - a0);
    const unsigned bytes = (unsigned)(((G * TW + skip + 1) & ~1) * 8);
    const unsigned long long* sl = s_slots + skip;
    T val[MS];
    unsigned long long t0 = 0;
    for (int it = 0;; ++it) {
        if (lane == 0) {
            mbar_arrive_expect(mbar, bytes);
            bulk_g2s(s_slots, tags + a0, bytes, mbar);
        }
        // one decision for the warp (a lane's own wait could end just past the limit)
        const bool got = __all_sync(0xffffffffu, mbar_wait_bounded(mbar, phase & 1u, tmo));
        phase++;
        if (!got) {
            mbar_wait_bounded(mbar, (phase - 1) & 1u, tmo);
            if (lane == 0) atomicExch(&bar->err, 1);
            return false;
        }
        bool ready = true;
#pragma unroll
        for (int m = 0; m < MS; ++m) {
            val[m] = T(0);
            if (lane + 32 * m < G && !tag_read_smem(sl + (int64_t)(lane + 32 * m) * TW, seq, &val[m])) ready = false;
        }
        __syncwarp();  // every lane has read the buffer before the next copy overwrites it
        if (__all_sync(0xffffffffu, ready)) break;
        int stop = 0;
        if (lane == 0) {
            const unsigned long long now = globaltimer_ns();
            if (it == 0) t0 = now;
            if (now - t0 > tmo) {
                atomicExch(&bar->err, 1);
                stop = 1;
            } else if ((it & 63) == 63 && *(volatile int*)&bar->err) {
                stop = 1;
            }
        }
        if (__shfl_sync(0xffffffffu, stop, 0)) return false;
    }
    T t = T(0);
#pragma unroll
    for (int m = 0; m < MS; ++m)
        if (lane + 32 * m < G) t = tag_add(t, val[m]);
    *total = warp_sum(t);
    return true;
}

// Warp 0 polls the slots of `set` (tag_poll_warp), then every thread gets the
// total; *s_ok = 0 after a timeout.  G: the blocks that publish (default: all).
template <typename T>
__device__ __forceinline__ T tag_wait(const unsigned long long* tags, int set, unsigned seq, GridBar* bar,
                                      unsigned long long tmo, T* s_tot, int* s_ok, int G = -1) {
    if (G < 0) G = gridDim.x;
    if (threadIdx.x < 32) {
        T t;
        const bool ok = tag_poll_warp<T>(tags, set, seq, G, bar, tmo, &t);
        if (threadIdx.x == 0) {
            *s_tot = t;
            *s_ok = ok ? 1 : 0;
        }
    }
    __syncthreads();
    return *s_tot;
}


// tag_wait with warp 0 polling by bulk copies (tag_poll_warp_bulk) when `bulk`,
// else by loads (tag_poll_warp): the same total either way.  The copy engine's
// round trip is the longer one, so it pays only where the pass's own loads
// would hold up a load poll.
template <typename T>
__device__ __forceinline__ T tag_wait_bulk(const unsigned long long* tags, int set, unsigned seq, GridBar* bar,
                                           unsigned long long tmo, T* s_tot, int* s_ok, int G,
                                           unsigned long long* s_slots, uint64_t* mbar, unsigned& phase,
                                           bool bulk) {
    if (threadIdx.x < 32) {
        T t;
        const bool ok = bulk ? tag_poll_warp_bulk<T>(tags, set, seq, G, bar, tmo, &t, s_slots, mbar, phase)
                             : tag_poll_warp<T>(tags, set, seq, G, bar, tmo, &t);
        if (threadIdx.x == 0) {
            *s_tot = t;
            *s_ok = ok ? 1 : 0;
        }
    }
    __syncthreads();
    return *s_tot;
}

}  // namespace bspai
