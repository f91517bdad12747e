// Batched dense contractions of the multipole method on the tensor cores (Section 3.1: the
// near-field tables of adjacent leaves and the translation operators M2L, P2M, P2L, L2P, M2P
// of the volume potential, and those of the double layer's multipole pass).
//
// A phase is a list of tasks y_t = T_op(t) x_t, T_op of size R x C (R, C <= 64), sorted by
// operator.  One CTA takes up to 128 tasks of one operator and forms them as one matrix product
// on the fifth-generation tensor cores:
//
//     D[m][n] = sum_k X[m][k] T[n][k],   m = task in the chunk (M = 128), n = output row
//     (N = R rounded up to 16), k = input column (K = C rounded up to 8),
//
// with tcgen05.mma kind::f16 on bfloat16 operands (binary32 accumulation in tensor memory).
// Every binary32 operand is split exactly into three bfloat16 parts, x = x1 + x2 + x3
// (x1 = x rounded to bfloat16, x2 = the remainder rounded, x3 = what is left; 3 x 8
// significant bits hold all 24 of binary32), and the product is formed as
//     X T ~ X1 T1 + X1 T2 + X2 T1 + X1 T3 + X2 T2 + X3 T1
// (six MMAs per K step; X1 T1 in one accumulator, the other five in a second one, added in
// the epilogue); the dropped terms X2 T3, X3 T2, X3 T3 are at most 2^-23 |X||T| per product,
// the size of binary32 rounding.  The operator's three parts are
// split once at set-up from the binary64 operator and stored in the exact shared-memory image
// the MMA reads, so a CTA stages it with one bulk copy; the sources are gathered, split and
// written into their images by all threads.
//
// Shared-memory images use the no-swizzle K-major layout of the tensor cores: core matrices of
// 8 rows x 16 bytes (8 x 8 bfloat16), row r of a core matrix at byte 16 r; the core matrix of
// rows 8g..8g+7 and columns 8c..8c+7 starts at byte c * LBO + g * 128 (SBO = 128 between row
// groups, LBO = rows * 16 between column groups).  One MMA consumes K = 16 columns (two column
// groups).
//
// Products leave tensor memory through tcgen05.ld (warp w reads lanes 32 (w % 4) .. + 31, i.e.
// tasks, and half w / 4 of the columns) and are written to the task-indexed product buffer
// (later summed per destination in a fixed order) or, in phases with one task per destination,
// straight to the destination.  Every wait on an mbarrier is bounded; a wait that gives up sets
// the error word, skips the rest of the work, waits (bounded) for its bulk copy and frees the
// tensor memory it holds.
#include <cuda_bf16.h>

#include <cstring>

#include "mh_internal.cuh"

namespace {

constexpr int TC_M = 128;         // tasks per CTA (rows of the MMA)
constexpr int TC_THREADS = 512;   // 16 warps: gather, epilogue (4 lane quarters x 4 column groups), output
constexpr unsigned TC_SPIN = 1u << 22;   // polls of an mbarrier before a wait gives up
constexpr int GATHER_MAX = TC_M * (64 / 8) / TC_THREADS;   // gather items per thread and part (K <= 64)

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor (tcgen05): start address, leading (K direction) and stride
// (row-group direction) byte offsets, all >> 4; descriptor version 1 at bits 46-47; no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: D binary32 (bits 4-5 = 1), A and B bfloat16 (bits 7-9
// and 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__device__ __forceinline__ uint32_t instr_desc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, P;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase `parity` of an mbarrier: true when it completed.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (unsigned i = 0; i < TC_SPIN; ++i)
        if (mbar_try_wait(mbar, parity)) return true;
    return false;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

// 16-byte asynchronous copy global -> shared; src_bytes = 0 fills the 16 bytes with zeros.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Exact split of a binary32 value into three bfloat16 parts (round to nearest even each time):
// x = p0 + p1 + p2 for every finite x whose parts stay in the normal range.
__device__ __forceinline__ void split3(float x, __nv_bfloat16& p0, __nv_bfloat16& p1, __nv_bfloat16& p2) {
    p0 = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(p0);
    p1 = __float2bfloat16_rn(r1);
    p2 = __float2bfloat16_rn(r1 - __bfloat162float(p1));
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// Byte offset of element (row, k) in a no-swizzle K-major bfloat16 image with `rows` rows.
__host__ __device__ __forceinline__ uint32_t img_off(int row, int k, int rows) {
    return (uint32_t)((k >> 3) * (rows * 16) + (row >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// Row stride of the product staging tile: R itself when R is odd (the lanes of a warp, which
// hold different rows, then hit distinct banks, and the tile is laid out like the product
// block), R + 1 otherwise.
__host__ __device__ __forceinline__ int stage_ld(int R) { return (R & 1) ? R : R + 1; }

// Products of a chunk (nt tasks from t0) from the staging tile to global memory.
//   temp form: one contiguous block temp[t0 R .. (t0 + nt) R); with stride R the tile is the
//   block itself and is copied with aligned 16-byte stores;
//   task_dst form: row t to dst[task_dst[t] ..], added when accumulate is set.
template <typename TD>
__device__ __forceinline__ void write_products(const float* __restrict__ stage_out, int ld, int R, int t0, int nt,
                                               float* __restrict__ temp, const int64_t* __restrict__ task_dst,
                                               int accumulate, TD* dst) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (!task_dst) {
        float* out = temp + (int64_t)t0 * R;
        const int ne = nt * R;
        if (ld == R) {
            // head up to a 16-byte boundary, aligned body, tail
            const int head = min(ne, (int)((4 - ((reinterpret_cast<uintptr_t>(out) >> 2) & 3)) & 3));
            if ((int)threadIdx.x < head) out[threadIdx.x] = stage_out[threadIdx.x];
            const int nb = (ne - head) >> 2;
            float4* o4 = reinterpret_cast<float4*>(out + head);
            for (int b = threadIdx.x; b < nb; b += TC_THREADS) {
                const float* sp = stage_out + head + 4 * b;
                o4[b] = make_float4(sp[0], sp[1], sp[2], sp[3]);
            }
            for (int e = head + 4 * nb + threadIdx.x; e < ne; e += TC_THREADS) out[e] = stage_out[e];
        } else {
            const int dr = TC_THREADS % R, dm = TC_THREADS / R;
            int mm = threadIdx.x / R, rr = threadIdx.x - mm * R;
            for (int e = threadIdx.x; e < ne; e += TC_THREADS) {
                out[e] = stage_out[mm * ld + rr];
                rr += dr;
                mm += dm;
                if (rr >= R) {
                    rr -= R;
                    ++mm;
                }
            }
        }
    } else {
        for (int mm = warp; mm < nt; mm += TC_THREADS / 32) {
            TD* y = dst + task_dst[t0 + mm];
            for (int rr = lane; rr < R; rr += 32) {
                const float v = stage_out[mm * ld + rr];
                y[rr] = accumulate ? y[rr] + (TD)v : (TD)v;
            }
        }
    }
}

// One CTA per chunk of up to 128 tasks of one operator (see the file comment).
//   img: operator images (parts 1, 2, 3, each npad x kpad bfloat16 in the layout above) at
//        img_off_op[op] (bfloat16 elements); kpad[op]: the operator's K extent (C rounded up to
//        16); op_C[op]: its columns C; R: rows (outputs) of every operator of the phase, npad =
//        R rounded up to 16; kmax: the largest kpad of the phase (sizes the source images);
//   src: binary32 pool (sources at task_src[t]); temp: products [task][R] unless task_dst is
//   given, then the products go to dst[task_dst[t] + r] (added when accumulate is set; TD =
//   float for the expansion pool, double for the potentials).
template <typename TD>
__global__ void __launch_bounds__(TC_THREADS, 2) k_contract_tc(
    const __nv_bfloat16* __restrict__ img, const int64_t* __restrict__ img_off_op, const int32_t* __restrict__ kpad_op,
    const int32_t* __restrict__ op_C, const int32_t* __restrict__ chunk_op, const int32_t* __restrict__ chunk_t0,
    const uint16_t* __restrict__ spl, int64_t plane, const int64_t* __restrict__ tc_src, int R, int npad, int kmax,
    float* __restrict__ temp, const int64_t* __restrict__ task_dst, int accumulate, TD* dst, int* err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // 1024-byte aligned base (the dynamic allocation is padded by 1 KB for this)
    unsigned char* base = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    const int a_bytes = TC_M * kmax * 2;        // one source image (one part)
    unsigned char* sA = base;                   // parts 1, 2, 3 of the sources
    unsigned char* sB = sA + 3 * a_bytes;       // parts 1, 2, 3 of the operator, 3 npad kpad bf16
    __shared__ __align__(8) uint64_t bar_copy, bar_mma;
    __shared__ uint32_t tmem_base;
    __shared__ int ok;

    const int ch = blockIdx.x;
    const int op = chunk_op[ch];
    const int t0 = chunk_t0[ch];
    const int nt = chunk_t0[ch + 1] - t0;
    const int C = op_C[op];
    const int kp = kpad_op[op];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // two accumulators of npad columns: the leading products X1 T1 at column 0, the five
    // smaller ones at column npad (a power of two >= 32 columns in all, npad <= 64)
    const uint32_t ncols = 2 * npad <= 32 ? 32u : 2 * npad <= 64 ? 64u : 128u;
    const uint32_t mb_copy = smem_addr(&bar_copy), mb_mma = smem_addr(&bar_mma);
    const uint32_t part_b = (uint32_t)(npad * kp * 2);   // bytes of one operator part

    if (threadIdx.x == 0) {
        mbar_init(mb_copy, 1);
        mbar_init(mb_mma, 1);
        fence_mbar_init();
        ok = 1;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = tmem_base;

    // the operator image: one bulk copy (16-byte aligned source and size)
    if (threadIdx.x == 0) {
        mbar_expect_tx(mb_copy, 3 * part_b);
        bulk_g2s(smem_addr(sB), img + img_off_op[op], 3 * part_b, mb_copy);
    }
    // the sources: already split into three bfloat16 planes with 16-element rows (tc_split),
    // so the gather is 16-byte asynchronous copies (8 columns of one part of one row each;
    // rows past the chunk are zero-filled).  Consecutive threads take 8 rows of one column
    // group, which fill one 128-byte line of the image: no bank conflicts.  A thread handles
    // the same (row, column group) items in every part; their row offsets are read first,
    // together, so the copies wait for one memory latency, not one per item.
    {
        const int groups = kp >> 3;
        int64_t roff[GATHER_MAX];
        uint32_t soff[GATHER_MAX];
        int nit = 0;
        {
            const int q = threadIdx.x >> 3;
            int rg = q / groups, cg = q - rg * groups;
            const int dq = (TC_THREADS >> 3) / groups, dc = (TC_THREADS >> 3) % groups;
#pragma unroll
            for (int it = 0; it < GATHER_MAX; ++it) {
                const int e = threadIdx.x + it * TC_THREADS;
                const int m = rg * 8 + (threadIdx.x & 7);
                roff[it] = e < TC_M * groups && m < nt ? tc_src[t0 + m] + 8 * cg : -1;
                soff[it] = img_off(m & (TC_M - 1), 8 * cg, TC_M);
                nit += e < TC_M * groups;
                rg += dq;
                cg += dc;
                if (cg >= groups) {
                    cg -= groups;
                    ++rg;
                }
            }
        }
        for (int part = 0; part < 3; ++part)
#pragma unroll
            for (int it = 0; it < GATHER_MAX; ++it)
                if (it < nit)
                    cp_async16(smem_addr(sA + part * a_bytes + soff[it]),
                               roff[it] >= 0 ? spl + part * plane + roff[it] : spl, roff[it] >= 0 ? 16u : 0u);
        asm volatile("cp.async.wait_all;" ::: "memory");
    }
    fence_async_smem();   // the generic-proxy stores above become visible to the tensor cores
    __syncthreads();

    if (threadIdx.x == 0) {
        if (!mbar_wait(mb_copy, 0)) {
            ok = 0;
            atomicExch(err, 1);
        } else {
            tc_after_sync();
            const uint32_t idesc = instr_desc_bf16(TC_M, npad);
            const uint32_t a_lbo = TC_M * 16, b_lbo = (uint32_t)npad * 16;
            const uint32_t a0 = smem_addr(sA), b0 = smem_addr(sB);
            // (source part, operator part) of the six products whose part indices sum to <= 2;
            // the first goes to the leading accumulator, the other five to the second.  The tensor
            // cores truncate when they add into an accumulator, so each accumulation costs up to
            // one unit in the last place of its running sum: the leading sum takes only K / 16 of
            // them, the second sum is ~2^-8 as large
            const int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {0, 1, 0, 2, 1, 0};
            for (int ks = 0; ks < kp / 16; ++ks) {
                const uint32_t da = (uint32_t)ks * 2 * a_lbo, db = (uint32_t)ks * 2 * b_lbo;
#pragma unroll
                for (int j = 0; j < 6; ++j)
                    mma_bf16(j == 0 ? tmem : tmem + (uint32_t)npad, smem_desc(a0 + pa[j] * a_bytes + da, a_lbo, 128),
                             smem_desc(b0 + pb[j] * part_b + db, b_lbo, 128), idesc,
                             j == 0 ? ks != 0 : (ks != 0 || j != 1));
            }
            mma_commit(mb_mma);
        }
    }
    // thread 0 waits for the products (the others wait at the barrier, without issuing); the
    // CTA goes on only if they came (the loads below are warp-collective)
    bool mine = true;
    if (threadIdx.x == 0) mine = ok && mbar_wait(mb_mma, 0);
    const bool have = __syncthreads_and(mine) != 0;
    const bool copied = ok != 0;
    if (copied && !have && threadIdx.x == 0) atomicExch(err, 2);
    tc_after_sync();
    // products: TMEM -> shared staging rows (stride stage_ld(R)) -> global, as whole rows
    float* stage = reinterpret_cast<float*>(sA);   // the source images are no longer read
    const int ld = stage_ld(R);
    if (have) {
        // warp w: tasks 32 (w % 4) + lane, column octets h, h + CG, ... (h = w / 4, CG =
        // TC_THREADS / 128 column groups)
        const int m = 32 * (warp & 3) + lane;
        const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
        for (int cc = 8 * (warp >> 2); cc < npad; cc += 8 * (TC_THREADS / 128)) {
            uint32_t r[8], q[8];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                : "r"(trow + (uint32_t)cc));
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
                : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7])
                : "r"(trow + (uint32_t)(npad + cc)));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (cc + u < R) stage[m * ld + cc + u] = __uint_as_float(r[u]) + __uint_as_float(q[u]);
        }
    }
    __syncthreads();
    if (have) {
        write_products<TD>(stage, ld, R, t0, nt, temp, task_dst, accumulate, dst);
    } else if (threadIdx.x == 0 && !copied) {
        mbar_wait(mb_copy, 0);   // the copy may still be in flight: let it land (bounded)
    }
    tc_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

// Split `count` consecutive binary32 vectors of length len (src) into the three bfloat16
// planes (plane elements apart) at dst, each vector padded with zeros to S entries.
__global__ void k_split_pool(const float* __restrict__ src, int len, int64_t count, int S,
                             uint16_t* __restrict__ planes, int64_t plane, int64_t dst) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count * S) return;
    const int64_t v = i / S;
    const int e = (int)(i - v * S);
    __nv_bfloat16 p0, p1, p2;
    split3(e < len ? src[v * len + e] : 0.f, p0, p1, p2);
    planes[dst + i] = __bfloat16_as_ushort(p0);
    planes[plane + dst + i] = __bfloat16_as_ushort(p1);
    planes[2 * plane + dst + i] = __bfloat16_as_ushort(p2);
}

// Host: round a binary32 value to bfloat16 (nearest, ties to even); returns the 16-bit pattern
// and the rounded value in *back.
uint16_t host_bf16(float x, float* back) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    uint32_t r;
    if ((u & 0x7F800000u) == 0x7F800000u)
        r = u >> 16;   // inf / nan
    else
        r = (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
    const uint32_t b = r << 16;
    std::memcpy(back, &b, 4);
    return (uint16_t)r;
}

}  // namespace

int tc_pad_rows(int R) { return (R + 15) / 16 * 16; }
int tc_pad_cols(int C) { return (C + 15) / 16 * 16; }

// Three-part bfloat16 image of one R x C operator (row-major, binary64) in the layout of the
// file comment: out receives 3 * npad * kpad bfloat16 values (16-bit patterns), part p at
// p * npad * kpad.  Part 1 = the value rounded to bfloat16 (through binary32), parts 2 and 3 =
// the remainders, formed in binary64 and rounded.
void tc_operator_image(const double* op, int R, int C, int npad, int kpad, uint16_t* out) {
    const size_t n = (size_t)npad * kpad;
    std::memset(out, 0, 3 * n * sizeof(uint16_t));
    for (int r = 0; r < R; ++r)
        for (int k = 0; k < C; ++k) {
            const double a = op[(size_t)r * C + k];
            float b0, b1, b2;
            const uint16_t p0 = host_bf16((float)a, &b0);
            const uint16_t p1 = host_bf16((float)(a - (double)b0), &b1);
            const uint16_t p2 = host_bf16((float)(a - (double)b0 - (double)b1), &b2);
            const size_t o = img_off(r, k, npad) / 2;
            out[o] = p0;
            out[n + o] = p1;
            out[2 * n + o] = p2;
        }
}

// Dynamic shared memory of a launch: the source and operator images, or, if larger, the product
// staging rows that reuse them (128 x (npad + 1) binary32), plus 1 KB for the alignment.
size_t tc_smem_bytes(int npad, int kmax) {
    const size_t images = (size_t)(3 * TC_M + 3 * npad) * kmax * 2;
    const size_t stage = (size_t)TC_M * stage_ld(npad) * 4;
    return (images > stage ? images : stage) + 1024;
}

// Largest operator of the tensor-core form: 64 x 64 (R, C <= 64).
static const size_t TC_SMEM_MAX = tc_smem_bytes(64, 64);

mh_status tc_prepare(mh_ctx* ctx) {
    static bool done[64] = {};
    if (ctx->device >= 0 && ctx->device < 64 && done[ctx->device]) return MH_OK;
    int optin = 0;
    MH_CUDA(ctx, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    cudaFuncAttributes fa{};
    MH_CUDA(ctx, cudaFuncGetAttributes(&fa, k_contract_tc<float>));
    if ((size_t)optin < TC_SMEM_MAX + fa.sharedSizeBytes)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "device shared memory (%d B per block) too small for the tensor-core "
                       "contraction (%zu B)", optin, TC_SMEM_MAX + fa.sharedSizeBytes);
    MH_CUDA(ctx, cudaFuncSetAttribute(k_contract_tc<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)TC_SMEM_MAX));
    MH_CUDA(ctx, cudaFuncSetAttribute(k_contract_tc<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)TC_SMEM_MAX));
    if (ctx->device >= 0 && ctx->device < 64) done[ctx->device] = true;
    return MH_OK;
}

mh_status tc_contract_launch(mh_ctx* ctx, const tc_launch& a) {
    const size_t smem = tc_smem_bytes(a.npad, a.kmax);
    if (smem > TC_SMEM_MAX || a.npad > 64 || a.kmax > 64)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "tensor-core contraction too large (%d x %d)", a.npad, a.kmax);
    if (a.n_chunks == 0) return MH_OK;
    if (a.dst_double)
        k_contract_tc<double><<<(unsigned)a.n_chunks, TC_THREADS, smem, ctx->stream>>>(
            reinterpret_cast<const __nv_bfloat16*>(a.img), a.img_off, a.kpad, a.op_C, a.chunk_op, a.chunk_t0, a.spl,
            a.plane, a.tc_src, a.R, a.npad, a.kmax, a.temp,
            a.task_dst, a.accumulate, static_cast<double*>(a.dst), a.err);
    else
        k_contract_tc<float><<<(unsigned)a.n_chunks, TC_THREADS, smem, ctx->stream>>>(
            reinterpret_cast<const __nv_bfloat16*>(a.img), a.img_off, a.kpad, a.op_C, a.chunk_op, a.chunk_t0, a.spl,
            a.plane, a.tc_src, a.R, a.npad, a.kmax, a.temp,
            a.task_dst, a.accumulate, static_cast<float*>(a.dst), a.err);
    MH_LAUNCHED(ctx);
    return MH_OK;
}

mh_status tc_split_launch(mh_ctx* ctx, const float* src, int len, int64_t count, int S, uint16_t* planes, int64_t plane,
                          int64_t dst) {
    if (count <= 0) return MH_OK;
    k_split_pool<<<(unsigned)mh_grid(count * S, 256), 256, 0, ctx->stream>>>(src, len, count, S, planes, plane, dst);
    MH_LAUNCHED(ctx);
    return MH_OK;
}
