// Fused x and y passes, FP32, N = 16 E1 (E1 in {4, 6, 8, 10, 12, 16}).
//
// Same operations as the separate passes (Sec. 2: the zero-padded transforms of the x and y
// axes on the way in, their inverses and the crop on the way out), in one persistent kernel
// per direction so that the intermediate array (x spectrum per plane, N rows of N+1 bins)
// never travels to HBM: it passes through a ring of R plane slots that stays in L2.
//
//   k_xy_fwd:  producer tasks  x forward of 32 rows of plane P  (rho -> ring slot P mod R)
//              consumer tasks  y forward of a 16-column tile of plane P  (ring -> w2)
//   k_yx_inv:  producer tasks  y inverse of a 16-column tile of plane P  (w3 -> ring slot)
//              consumer tasks  x inverse of 32 rows of plane P  (ring -> u)
//
// The task bodies are those of the warp forms (xw_fwd_pair / xw_inv_pair for a row pair per
// half-warp, yw_* for a column pair per warp).  CTAs take tasks in one global order from an
// atomic counter: the producers of plane s, then the consumers of plane s - D, for
// s = 0, 1, ...  A consumer of plane P waits until every producer of P has finished
// (per-slot completion counters, release / acquire at GPU scope); a producer of plane P
// waits until every consumer of plane P - R, the slot's previous tenant, has finished.  Both
// dependencies come earlier in the order (R > D), and a CTA only waits on tasks taken before
// its own, so the oldest unfinished task can always run and the pass finishes whatever
// number of CTAs is resident.  Every wait is bounded; on a timeout the status word records
// it and the kernel runs on, so it still ends.  The last CTA to leave returns the counters
// to zero for the next launch.
#pragma once
#include "passes_zwarp.cuh"

namespace gsp {

// Largest ring (plane slots) a fused pass uses; the counter block holds 2 + 2 kRingMax ints.
constexpr int kRingMax = 256;
constexpr int kSyncInts = 2 + 2 * kRingMax;
// Polls of a completion counter (each followed by a sleep of at least 256 ns) before a
// wait gives up.
constexpr long long kCounterWaitLimit = 1ll << 20;

__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_gpu(int *p, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Order generic-proxy accesses of global memory with async-proxy (TMA) ones.
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Bounded wait until *p >= target (acquire).  Once any wait of the plan has given up (the
// timeout bit of *status), later ones return at once, so that a failed pass ends after one
// wait limit instead of one per dependent task.
__device__ __forceinline__ void counter_wait(const int *p, int target, int *status) {
    for (long long it = 0; it < kCounterWaitLimit; ++it) {
        if (ld_acquire_gpu(p) >= target) return;
        if (*reinterpret_cast<volatile int *>(status) & kStatusTimeout) return;
        __nanosleep(256);
    }
    atomicOr(status, kStatusTimeout);
}

// Task order of a fused pass over P planes: step s holds the NA producer tasks of plane s
// (s < P) and then the NB consumer tasks of plane s - D (s >= D).
struct XYOrder {
    int P, D, NA, NB;
    __device__ __forceinline__ int count() const { return P * (NA + NB); }
    // kind 0: producer, 1: consumer.
    __device__ __forceinline__ void task(int t, int &kind, int &plane, int &idx) const {
        const int A = D * NA;
        if (t < A) {
            kind = 0, plane = t / NA, idx = t % NA;
            return;
        }
        t -= A;
        const int S = NA + NB, M = (P - D) * S;
        if (t < M) {
            const int s = D + t / S, r = t % S;
            if (r < NA) kind = 0, plane = s, idx = r;
            else kind = 1, plane = s - D, idx = r - NA;
            return;
        }
        t -= M;
        kind = 1, plane = P - D + t / NB, idx = t % NB;
    }
};

template <int E1> struct XYWarp {
    static constexpr int N = 16 * E1, H = E1 / 2, NT = 256, TC = 16;
    static constexpr int NX = N / 32;                 // x tasks per plane (a row pair per half-warp)
    static constexpr int NY = (N + 1 + TC - 1) / TC;  // y tasks per plane (16-column tiles)
    static constexpr int T_BYTES = E1 * 32 * 8, TX_BYTES = N * 8, T2_BYTES = (N / 2 + 1) * 8;
    // Forward: the y task's input tile (N rows x 128 B), its exchange / output tile (2N rows,
    // also the x tasks' 16 x 4 KB half-warp slots), the tables, one mbarrier, two task slots.
    static constexpr int F_IN = 0, F_XB = (N * 128 + 1023) / 1024 * 1024, F_T = F_XB + 65536;
    static constexpr int F_TX = F_T + T_BYTES, F_T2 = F_TX + TX_BYTES;
    static constexpr int F_BAR = (F_T2 + T2_BYTES + 15) / 16 * 16, SMEM_F = 1024 + F_BAR + 64;
    // Inverse: one 64 KB tile (2N input rows, exchange, N output rows; the x tasks' slots).
    static constexpr int I_XB = 0, I_T = 65536, I_TX = I_T + T_BYTES, I_T2 = I_TX + TX_BYTES;
    static constexpr int I_BAR = (I_T2 + T2_BYTES + 15) / 16 * 16, SMEM_I = 1024 + I_BAR + 64;
    static_assert(N % 32 == 0 && NY * TC <= ((N + 1 + 15) / 16) * 16, "tiles stay inside the row pitch");
};

// Shared prologue / epilogue of both directions.
__device__ __forceinline__ void xy_exit(int *sync, int R) {
    // Every CTA has taken its last task index and sent its last completion before it
    // counts itself out; the last one resets the block for the next launch.
    __threadfence();
    if (atomicAdd(sync + 1, 1) == (int)gridDim.x - 1) {
        __threadfence();
        for (int i = 0; i < R; ++i) sync[2 + i] = sync[2 + kRingMax + i] = 0;
        sync[0] = 0;
        sync[1] = 0;
        __threadfence();
    }
}

template <int E1>
__global__ void __launch_bounds__(XYWarp<E1>::NT, 2)
k_xy_fwd(const PtrArray rho, float2 *__restrict__ ring, const __grid_constant__ CUtensorMap tring,
         const __grid_constant__ CUtensorMap tout, const float2 *__restrict__ tw, const XYOrder ord, int R, int Px,
         int *__restrict__ sync, int *__restrict__ status) {
    using X = XYWarp<E1>;
    constexpr int N = X::N, H = X::H, NX = X::NX, NY = X::NY;
    extern __shared__ __align__(16) unsigned char smraw[];
    griddep_wait();  // the previous kernel has finished (and reset the counter block)
    unsigned char *base = smraw + ((1024 - (smem_addr(smraw) & 1023)) & 1023);
    unsigned char *inb = base + X::F_IN, *xb = base + X::F_XB;
    float2 *T = reinterpret_cast<float2 *>(base + X::F_T);
    float2 *TX = reinterpret_cast<float2 *>(base + X::F_TX);
    float2 *T2 = reinterpret_cast<float2 *>(base + X::F_T2);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + X::F_BAR);
    volatile int *next = reinterpret_cast<volatile int *>(bar + 1);
    int *prod = sync + 2, *cons = sync + 2 + kRingMax;
    const int ntasks = ord.count();
    const int g = threadIdx.x >> 5, q = threadIdx.x & 31, hw = threadIdx.x >> 4, qq = q & 15;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        next[0] = atomicAdd(sync, 1);
    }
    for (int i = threadIdx.x; i < E1 * 32; i += X::NT) T[i] = tw[(i & 31) * (i >> 5)];
    xw_tables<N>(TX, T2, tw);
    __syncthreads();
    const ZwLane zl = zw_lane<E1>(tw, smem_addr(xb), g, q);
    const int io = zw_sw128(q, g);
    const int kb = (q & 7) + H * ((q >> 3) & 1) + E1 * (q >> 4);
    const uint32_t xs = smem_addr(xb) + 4096 * hw;
    uint32_t ph = 0;
    for (int it = 0;; ++it) {
        const int t = next[it & 1];
        if (t >= ntasks) break;
        if (threadIdx.x == 0) next[(it + 1) & 1] = atomicAdd(sync, 1);
        int kind, P, idx;
        ord.task(t, kind, P, idx);
        const int slot = P % R, epoch = P / R;
        if (kind == 0) {
            // x forward of rows 32 idx .. 32 idx + 31 of plane P into the slot, once the y
            // tasks of the slot's previous plane have read it.
            if (threadIdx.x == 0 && epoch > 0) counter_wait(cons + slot, epoch * NY, status);
            __syncthreads();
            float2 f[2 * H];
            xw_load<N>(rho, P * (N / 2) + 16 * idx + hw, qq, f);
            float2 *d0 = ring + ((long long)slot * N + 32 * idx + 2 * hw) * Px;
            xw_fwd_pair<N>(f, xs, qq, TX, T2, d0, d0 + Px);
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                fence_proxy_async_global();
                red_release_gpu(prod + slot, 1);
            }
        } else {
            // y forward of the 16-column tile idx of plane P, ring -> w2.
            if (threadIdx.x == 0) {
                counter_wait(prod + slot, (epoch + 1) * NX, status);
                fence_proxy_async_global();
                mbar_arrive_expect_tx(bar, N * 128);
                tma_load_3d(inb, &tring, bar, idx * X::TC, 0, slot);
            }
            // The rest of warp 0 waits here, not in the mbarrier poll below, while thread 0
            // waits for the producers: no spin of a diverged part of the warp on another.
            __syncwarp();
            const bool ok = mbar_wait(bar, ph, status);
            ph ^= 1;
            if (threadIdx.x == 0) red_release_gpu(cons + slot, 1);  // the slot's tile is in shared memory
            if (ok && idx * X::TC + 2 * g < N + 1) {
                CV v[16];
                yw_fwd_front<E1, 128>(v, inb, io, zl, T);
                yw_fwd_back<E1, 128>(v, zl, xb, kb, g);
            }
            fence_proxy_async();
            __syncthreads();
            if (threadIdx.x == 0) {
                tma_store_3d(&tout, xb, idx * X::TC, 0, P);
                tma_store_3d(&tout, xb + N * 128, idx * X::TC, N, P);
                bulk_commit();
                bulk_wait_read0();
            }
        }
        __syncthreads();  // next task index published; xb and inb free
    }
    if (threadIdx.x == 0) {
        bulk_wait0();
        xy_exit(sync, R);
    }
}

template <int E1>
__global__ void __launch_bounds__(XYWarp<E1>::NT, 2)
k_yx_inv(const __grid_constant__ CUtensorMap tin, float2 *__restrict__ ring, const PtrArray u,
         const float2 *__restrict__ tw, const XYOrder ord, int R, int Px, int *__restrict__ sync,
         int *__restrict__ status) {
    using X = XYWarp<E1>;
    constexpr int N = X::N, H = X::H, NX = X::NX, NY = X::NY, NN = N * N;
    extern __shared__ __align__(16) unsigned char smraw[];
    griddep_wait();  // the previous kernel has finished (and reset the counter block)
    unsigned char *base = smraw + ((1024 - (smem_addr(smraw) & 1023)) & 1023);
    unsigned char *xb = base + X::I_XB;
    float2 *T = reinterpret_cast<float2 *>(base + X::I_T);
    float2 *TX = reinterpret_cast<float2 *>(base + X::I_TX);
    float2 *T2 = reinterpret_cast<float2 *>(base + X::I_T2);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + X::I_BAR);
    volatile int *next = reinterpret_cast<volatile int *>(bar + 1);
    int *prod = sync + 2, *cons = sync + 2 + kRingMax;
    const int ntasks = ord.count();
    const int g = threadIdx.x >> 5, q = threadIdx.x & 31, hw = threadIdx.x >> 4, qq = q & 15;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        next[0] = atomicAdd(sync, 1);
    }
    for (int i = threadIdx.x; i < E1 * 32; i += X::NT) T[i] = tw[(i & 31) * (i >> 5)];
    xw_tables<N>(TX, T2, tw);
    __syncthreads();
    const uint32_t xs = smem_addr(xb) + 4096 * hw;
    uint32_t ph = 0;
    for (int it = 0;; ++it) {
        const int t = next[it & 1];
        if (t >= ntasks) break;
        if (threadIdx.x == 0) next[(it + 1) & 1] = atomicAdd(sync, 1);
        int kind, P, idx;
        ord.task(t, kind, P, idx);
        const int slot = P % R, epoch = P / R;
        if (kind == 0) {
            // y inverse of the 16-column tile idx of plane P, w3 -> the slot, once the x tasks
            // of the slot's previous plane have read it.
            if (threadIdx.x == 0) {
                mbar_arrive_expect_tx(bar, 2 * N * 128);
                tma_load_3d(xb, &tin, bar, idx * X::TC, 0, P);
                tma_load_3d(xb + N * 128, &tin, bar, idx * X::TC, N, P);
            }
            const bool ok = mbar_wait(bar, ph, status);
            ph ^= 1;
            if (ok && idx * X::TC + 2 * g < N + 1) {
                // Lane constants of the y form, made here so that they do not stay live
                // through the x tasks.
                const ZwLane zl = zw_lane<E1>(tw, smem_addr(xb), g, q);
                const int kb = (q & 7) + H * ((q >> 3) & 1) + E1 * (q >> 4);
                CV v[16];
                yw_inv<E1, 128>(v, zl, xb, kb, zw_sw128(q, g), g, T);
            }
            if (threadIdx.x == 0 && epoch > 0) counter_wait(cons + slot, epoch * NX, status);
            __syncthreads();
            // The N output rows (16 columns of 8 bytes each) to the slot: thread t copies the
            // 16-byte chunk t % 8 of rows t / 8 + 32 j, coalesced 128-byte row segments.
            {
                const int c = threadIdx.x & 7;
                float2 *dst = ring + (long long)slot * N * Px + idx * X::TC + 2 * c;
#pragma unroll 4
                for (int y = threadIdx.x >> 3; y < N; y += X::NT / 8)
                    __stcg(reinterpret_cast<float4 *>(dst + (long long)y * Px),
                           *reinterpret_cast<const float4 *>(xb + zw_sw128(y, c)));
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                red_release_gpu(prod + slot, 1);
            }
        } else {
            // x inverse of rows 32 idx .. 32 idx + 31 of plane P, the slot -> u.
            if (threadIdx.x == 0) counter_wait(prod + slot, (epoch + 1) * NY, status);
            __syncthreads();
            const int i = P * (N / 2) + 16 * idx + hw;
            const float2 *s0 = ring + ((long long)slot * N + 32 * idx + 2 * hw) * Px;
            const int b = (2 * i) / NN;
            float2 *d = reinterpret_cast<float2 *>(const_cast<void *>(u.p[b])) + (long long)(2 * i - b * NN) * (N / 2) + qq;
            xw_inv_pair<N, true, 3>(s0, s0 + Px, xs, qq, TX, T2, d);
            __syncthreads();
            if (threadIdx.x == 0) red_release_gpu(cons + slot, 1);  // its rows have been read
        }
        fence_proxy_async();  // this task's generic writes of xb before the next TMA load into it
        __syncthreads();      // next task index published; xb free
    }
    if (threadIdx.x == 0) xy_exit(sync, R);
}

}  // namespace gsp
