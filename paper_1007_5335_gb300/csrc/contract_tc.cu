// Batched dense contractions of the multipole method on the tensor cores (Section 3.1: the
// near-field tables of adjacent leaves and the translation operators M2L, P2M, P2L, L2P, M2P
// of the volume potential, and those of the double layer's multipole pass).
//
// A phase is a list of tasks y_t = T_op(t) x_t, T_op of size R x C (R, C <= 64), sorted by
// operator and cut into chunks of up to 128 tasks of one operator.  A chunk is one matrix
// product on the fifth-generation tensor cores:
//
//     D[m][n] = sum_k X[m][k] T[n][k],   m = task in the chunk (M = 128), n = output row
//     (N = R rounded up to 16), k = input column (K = C rounded up to 16),
//
// with tcgen05.mma kind::f16 on bfloat16 operands (binary32 accumulation in tensor memory).
// Every binary32 operand is split exactly into three bfloat16 parts, x = x1 + x2 + x3
// (x1 = x rounded to bfloat16, x2 = the remainder rounded, x3 = what is left; 3 x 8
// significant bits hold all 24 of binary32), and the product is formed as
//     X T ~ X1 T1 + (X1 T2 + X2 T1) + (X2 T2 + X1 T3 + X3 T1);
// the dropped terms X2 T3, X3 T2, X3 T3 are at most 2^-23 |X||T| per product, the size of
// binary32 rounding.  An MMA instruction costs about the same whatever its N (up to 256), so
// the operator's three parts are stacked along N and four MMAs per K step form the products:
// X1 [T1; T2] and X2 [T1; T2] (N = 2 npad), then X1 T3 and X3 T1 (N = npad), both added into
// the X2 T2 block.  The leading products X1 T1 keep an accumulator
// block of their own; the blocks are added in the epilogue, smallest first.  The operator's
// parts are split once at set-up from the binary64 operator and stored in the exact
// shared-memory image the MMAs read, so it is staged by one bulk copy; the sources are split by
// the kernel that finalises them (k_split_pool) and gathered into their images by 16-byte
// asynchronous copies.
//
// The kernel is persistent and warp-specialised: one CTA per SM takes a contiguous range of
// chunks (neighbouring chunks often share their operator, whose image then stays in place) and
// runs them through a pipeline of shared-memory stages and two tensor-memory accumulator sets:
//   producer warps: wait until a stage is free, copy the operator image (one bulk copy,
//     skipped when the stage holds it already) and gather the sources of the next chunk into it;
//   MMA warp (one thread): once a stage is full and an accumulator set free, issue the chunk's
//     MMAs; their completion frees the stage and fills the accumulator set;
//   epilogue warps: move the products out of tensor memory into a shared staging tile (which
//     frees the accumulator set) and write them to global memory.
// So the gather of chunk j + 1 and the MMAs of chunk j + 1 run while the products of chunk j
// leave.  Synchronisation is by mbarriers only, except a named barrier among the epilogue warps.
//
// The operator image uses the no-swizzle K-major layout of the tensor cores: core matrices of
// 8 rows x 16 bytes (8 x 8 bfloat16), row r of a core matrix at byte 16 r; the core matrix of
// rows 8g..8g+7 and columns 8c..8c+7 starts at byte c * LBO + g * 128 (SBO = 128 between row
// groups, LBO = rows * 16 between column groups); the source images use the 128-byte swizzled
// K-major layout (smem_desc_sw128).  One MMA consumes K = 16 columns (two column
// groups).
//
// Products are written to the task-indexed product buffer (later summed per destination in a
// fixed order) or, in phases with one task per destination, straight to the destination.
// Every wait on an mbarrier is bounded and also ends when another role has given up: a wait
// that gives up sets the error word and a shared abort flag, every role then leaves its loop,
// in-flight copies and MMAs are waited for (bounded) and the tensor memory is freed.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "mh_internal.cuh"

namespace {

constexpr int TC_M = 128;                 // tasks per chunk (rows of the MMA)
constexpr int EPI_WARPS = 8;              // warps 0-7: epilogue (lane quarter w % 4, column octets w / 4 + 2 i)
constexpr int MMA_WARP = 8;               // warp 8: tensor memory and the MMAs (lane 0)
constexpr int PROD_WARPS = 4;             // warps 9-12: sources
constexpr int EPI_THREADS = 32 * EPI_WARPS;
constexpr int PROD0 = 32 * (EPI_WARPS + 1);             // first producer thread
constexpr int TC_THREADS = PROD0 + 32 * PROD_WARPS;     // 416
constexpr int TC_MAX_STAGES = 4;
constexpr unsigned TC_SPIN = 1u << 22;    // try_wait calls of an mbarrier before a wait gives up
static_assert(32 * PROD_WARPS == TC_M, "one producer thread per task row");

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor (tcgen05): start address, leading (K direction) and stride
// (row-group direction) byte offsets, all >> 4; descriptor version 1 at bits 46-47; no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Descriptor of a K-major operand in the 128-byte swizzled layout: rows of 128 bytes (64
// bfloat16 of K), 8-row groups of 1024 bytes (SBO), the 16-byte chunk c of row r stored at
// chunk c ^ (r % 8) of its row; layout type 2 at bits 61-63; the group must start on a 1024-byte
// boundary.  A later K step inside the row is reached by adding its byte offset / 16.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
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

// Bounded wait that also ends (false) once *abort is set by another role.
__device__ __forceinline__ bool mbar_wait_ab(uint32_t mbar, uint32_t parity, const volatile int* abort) {
    for (unsigned i = 0; i < TC_SPIN; ++i) {
        if (mbar_try_wait(mbar, parity)) return true;
        if (*abort) return false;
    }
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

// AND of `pred` over the `count` threads that meet at named barrier `id`.
__device__ __forceinline__ bool bar_and(bool pred, int id, int count) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void bar_named(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

// 16-byte asynchronous copy global -> shared through L2 only (the gathered rows are not reused
// by the SM); src_bytes = 0 fills the 16 bytes with zeros.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
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

// Byte offset of element (row, k) in a no-swizzle K-major bfloat16 image with `rows` rows.
__host__ __device__ __forceinline__ uint32_t img_off(int row, int k, int rows) {
    return (uint32_t)((k >> 3) * (rows * 16) + (row >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// One source image (one part): 128 rows of 128 bytes in the swizzled layout.
constexpr int A_PART = TC_M * 128;
// Bytes of one pipeline stage: three source images and the operator image (three parts of
// npad x kmax bfloat16), rounded up to 1024 so that every stage's images start on a 1024-byte
// boundary.
__host__ __device__ __forceinline__ int tc_stage_size(int npad, int kmax) {
    return (3 * A_PART + 3 * npad * kmax * 2 + 1023) / 1024 * 1024;
}

// Row stride of the product staging tile: R itself when R is odd (the lanes of a warp, which
// hold different rows, then hit distinct banks, and the tile is laid out like the product
// block), R + 1 otherwise.
__host__ __device__ __forceinline__ int stage_ld(int R) { return (R & 1) ? R : R + 1; }

// Products of a chunk (nt tasks from t0) from the staging tile (row stride ld) to global
// memory, by the NTH epilogue threads (thread index e < NTH):
//   temp form: one contiguous block temp[t0 R .. (t0 + nt) R); with stride R the tile is the
//   block itself and is copied with aligned 16-byte stores;
//   task_dst form: row t to dst[task_dst[t] ..], added when accumulate is set.  A warp takes
//   rows w, w + NTH/32, ...: it reads the destinations of 32 of them at once, then moves four
//   rows per round (loads of all four before their stores).
template <typename TD, int NTH>
__device__ __forceinline__ void write_products(const float* __restrict__ stage_out, int ld, int R, int t0, int nt,
                                               float* __restrict__ temp, const int64_t* __restrict__ task_dst,
                                               int accumulate, TD* dst, int e) {
    constexpr int NW = NTH / 32;
    const int warp = e >> 5, lane = e & 31;
    if (!task_dst) {
        float* out = temp + (int64_t)t0 * R;
        const int ne = nt * R;
        if (ld == R) {
            // head up to a 16-byte boundary, aligned body, tail
            const int head = min(ne, (int)((4 - ((reinterpret_cast<uintptr_t>(out) >> 2) & 3)) & 3));
            if (e < head) out[e] = stage_out[e];
            const int nb = (ne - head) >> 2;
            float4* o4 = reinterpret_cast<float4*>(out + head);
            for (int b = e; b < nb; b += NTH) {
                const float* sp = stage_out + head + 4 * b;
                o4[b] = make_float4(sp[0], sp[1], sp[2], sp[3]);
            }
            for (int q = head + 4 * nb + e; q < ne; q += NTH) out[q] = stage_out[q];
        } else {
            const int dr = NTH % R, dm = NTH / R;
            int mm = e / R, rr = e - mm * R;
            for (int q = e; q < ne; q += NTH) {
                out[q] = stage_out[mm * ld + rr];
                rr += dr;
                mm += dm;
                if (rr >= R) {
                    rr -= R;
                    ++mm;
                }
            }
        }
    } else {
        const int rows = nt > warp ? (nt - warp + NW - 1) / NW : 0;   // this warp's rows
        for (int i0 = 0; i0 < rows; i0 += 32) {
            const int cnt = min(32, rows - i0);
            const int64_t dl = lane < cnt ? task_dst[t0 + warp + NW * (i0 + lane)] : 0;
            for (int i1 = 0; i1 < cnt; i1 += 4) {
                TD* y[4];
                float v[4][2];
                TD old[4][2];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int64_t d = __shfl_sync(0xffffffffu, dl, min(i1 + k, cnt - 1));
                    const int mm = warp + NW * (i0 + i1 + k);
                    y[k] = i1 + k < cnt ? dst + d : nullptr;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int rr = lane + 32 * h;
                        v[k][h] = y[k] && rr < R ? stage_out[mm * ld + rr] : 0.f;
                        old[k][h] = y[k] && rr < R && accumulate ? y[k][rr] : (TD)0;
                    }
                }
#pragma unroll
                for (int k = 0; k < 4; ++k)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int rr = lane + 32 * h;
                        if (y[k] && rr < R) y[k][rr] = old[k][h] + (TD)v[k][h];
                    }
            }
        }
    }
}

// Persistent warp-specialised contraction (see the file comment).  CTA b takes chunks
// [n_chunks b / G, n_chunks (b + 1) / G), G = gridDim.x.
//   img: operator images (parts 1, 2, 3, each npad x kpad bfloat16 in the layout above) at
//        img_off_op[op] (bfloat16 elements); kpad[op]: the operator's K extent (its columns
//        rounded up to 16); R: rows (outputs) of every operator of the phase, npad = R rounded
//        up to 16; kmax: the largest kpad of the phase (sizes the stages); nst: stages (2..4);
//   spl: the three bfloat16 planes of the sources (plane elements apart), the source of task t
//        at tc_src[t] (rows padded with zeros to a multiple of 16 entries);
//   temp: products [task][R] unless task_dst is given, then the products go to
//   dst[task_dst[t] + r] (added when accumulate is set; TD = float for the expansion pool,
//   double for the potentials).
template <typename TD>
__global__ void __launch_bounds__(TC_THREADS, 1) k_contract_tc(
    const __nv_bfloat16* __restrict__ img, const int64_t* __restrict__ img_off_op, const int32_t* __restrict__ kpad_op,
    const int32_t* __restrict__ chunk_op, const int32_t* __restrict__ chunk_t0, int n_chunks,
    const uint16_t* __restrict__ spl, int64_t plane, const int64_t* __restrict__ tc_src, int R, int npad, int kmax,
    int nst, float* __restrict__ temp, const int64_t* __restrict__ task_dst, int accumulate, TD* dst, int* err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // 1024-byte aligned base (the dynamic allocation is padded by 1 KB for this)
    unsigned char* base = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    const int stage_bytes = tc_stage_size(npad, kmax);
    float* tile = reinterpret_cast<float*>(base + nst * stage_bytes);   // products, TC_M x stage_ld(R)
    __shared__ __align__(8) uint64_t full[TC_MAX_STAGES], opf[TC_MAX_STAGES], empty[TC_MAX_STAGES];
    __shared__ __align__(8) uint64_t accf[2], acce[2], fin;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ int stage_op[TC_MAX_STAGES];
    volatile int* ab = &abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c_begin = (int)((int64_t)n_chunks * blockIdx.x / gridDim.x);
    const int c_end = (int)((int64_t)n_chunks * (blockIdx.x + 1) / gridDim.x);
    // two accumulator sets of four blocks of npad columns (see the MMA warp)
    const uint32_t ncols = 8 * npad <= 128 ? 128u : 8 * npad <= 256 ? 256u : 512u;
    auto give_up = [&](int code) {
        atomicExch(err, code);
        *ab = 1;
    };

    if (threadIdx.x == 0) {
        for (int q = 0; q < nst; ++q) {
            mbar_init(smem_addr(&full[q]), 32 * PROD_WARPS);
            mbar_init(smem_addr(&opf[q]), 1);
            mbar_init(smem_addr(&empty[q]), 1);
            stage_op[q] = -1;
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(smem_addr(&accf[q]), 1);
            mbar_init(smem_addr(&acce[q]), EPI_THREADS);
        }
        mbar_init(smem_addr(&fin), 1);
        fence_mbar_init();
        abort_flag = 0;
    }
    if (warp == MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = tmem_base;

    if (warp > MMA_WARP) {
        // ---- producers: warp pw, lane (r8 = lane % 8, cq = lane / 8) copies rows
        //      8 (pw + 4 i) + r8 (i < 4), column groups cq and cq + 4, of every part: one warp
        //      instruction moves 64 contiguous bytes of each of 8 rows into 512 conflict-free
        //      bytes of shared memory ----
        const int pw = warp - (MMA_WARP + 1), r8 = lane & 7, cq = lane >> 3;
        const bool lead = threadIdx.x == PROD0;   // issues the operator copies
        int prev = -1;             // stage of the previous chunk (its copies are completed one chunk late)
        int last_j[TC_MAX_STAGES];  // lead: last chunk index per stage with a bulk copy
#pragma unroll
        for (int q = 0; q < TC_MAX_STAGES; ++q) last_j[q] = -1;
        // rolling prefetch of the chunk descriptions, so that no load waits inside an iteration:
        // (op, t0, t1) of chunk ch + 1 come from iteration ch - 1, its K extent and row offsets
        // from iteration ch
        int op = 0, t0 = 0, t1 = 0, kp = 0, op_n = 0, t0_n = 0, t1_n = 0;
        int64_t off[4], ioff = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) off[i] = -1;
        if (c_begin < c_end) {
            op = chunk_op[c_begin];
            t0 = chunk_t0[c_begin];
            t1 = chunk_t0[c_begin + 1];
            kp = kpad_op[op];
            ioff = img_off_op[op];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int m = 8 * (pw + 4 * i) + r8;
                off[i] = m < t1 - t0 ? tc_src[t0 + m] : -1;
            }
        }
        if (c_begin + 1 < c_end) {
            op_n = chunk_op[c_begin + 1];
            t0_n = chunk_t0[c_begin + 1];
            t1_n = chunk_t0[c_begin + 2];
        }
        int j = 0;
        for (int ch = c_begin; ch < c_end; ++ch, ++j) {
            int kp_n = 0, op_nn = 0, t0_nn = 0, t1_nn = 0;
            int64_t off_n[4], ioff_n = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) off_n[i] = -1;
            if (ch + 1 < c_end) {
                kp_n = kpad_op[op_n];
                ioff_n = img_off_op[op_n];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int m = 8 * (pw + 4 * i) + r8;
                    off_n[i] = m < t1_n - t0_n ? tc_src[t0_n + m] : -1;
                }
            }
            if (ch + 2 < c_end) {
                op_nn = chunk_op[ch + 2];
                t0_nn = chunk_t0[ch + 2];
                t1_nn = chunk_t0[ch + 3];
            }
            const int s = j % nst;
            if (j >= nst && !mbar_wait_ab(smem_addr(&empty[s]), (uint32_t)((j / nst) - 1) & 1u, ab)) {
                give_up(3);
                break;
            }
            unsigned char* sA = base + s * stage_bytes;
            if (lead) {
                const uint32_t bar = smem_addr(&opf[s]);
                if (stage_op[s] != op) {
                    const uint32_t bytes = (uint32_t)(3 * npad * kp * 2);
                    stage_op[s] = op;
                    mbar_expect_tx(bar, bytes);
                    bulk_g2s(smem_addr(sA + 3 * A_PART), img + ioff, bytes, bar);
#pragma unroll
                    for (int q = 0; q < TC_MAX_STAGES; ++q)
                        if (q == s) last_j[q] = j;
                } else {
                    mbar_arrive(bar);   // the stage holds this operator already
                }
            }
            // 16-byte copies (8 columns of one part of one row) into the swizzled images; rows
            // past the chunk are zero-filled; columns past kp are never read
            const __nv_bfloat16* dummy = img;   // any valid address for the zero-fill form
#pragma unroll
            for (int part = 0; part < 3; ++part)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int m = 8 * (pw + 4 * i) + r8;
#pragma unroll
                    for (int hcg = 0; hcg < 2; ++hcg) {
                        const int cg = cq + 4 * hcg;
                        if (cg < (kp >> 3))
                            cp_async16(smem_addr(sA + part * A_PART + m * 128 + ((cg ^ r8) << 4)),
                                       off[i] >= 0 ? static_cast<const void*>(spl + part * plane + off[i] + 8 * cg)
                                                   : static_cast<const void*>(dummy),
                                       off[i] >= 0 ? 16u : 0u);
                    }
                }
            cp_async_commit();
            if (prev >= 0) {
                // the previous chunk's copies have landed: make them visible to the tensor cores
                cp_async_wait_group<1>();
                fence_async_smem();
                mbar_arrive(smem_addr(&full[prev]));
            }
            prev = s;
            op = op_n;
            t0 = t0_n;
            t1 = t1_n;
            kp = kp_n;
#pragma unroll
            for (int i = 0; i < 4; ++i) off[i] = off_n[i];
            ioff = ioff_n;
            op_n = op_nn;
            t0_n = t0_nn;
            t1_n = t1_nn;
        }
        cp_async_wait_group<0>();
        if (prev >= 0) {
            fence_async_smem();
            mbar_arrive(smem_addr(&full[prev]));
        }
        if (lead && *ab) {
            // on the way out after a failure: let the bulk copies in flight land (bounded)
            for (int q = 0; q < nst; ++q)
                if (last_j[q] >= 0) mbar_wait(smem_addr(&opf[q]), (uint32_t)(last_j[q] / nst) & 1u);
        }
    } else if (warp == MMA_WARP) {
        // ---- MMA issue: one thread ----
        if (lane == 0) {
            // accumulator set a: four blocks of npad columns from column 4 a npad, X1 T1 | X1 T2 |
            // X2 T1 | X2 T2 + X1 T3 + X3 T1.  The tensor cores truncate when they add into an
            // accumulator (up to one unit in the last place of the running sum per addition): the
            // leading products keep a block of their own and the three smallest share one
            const uint32_t id2 = instr_desc_bf16(TC_M, 2 * npad), id1 = instr_desc_bf16(TC_M, npad);
            const uint32_t b_lbo = (uint32_t)npad * 48;   // the stacked image has 3 npad rows
            int j = 0;
            // rolling prefetch: the operator of chunk ch + 2 and the K extent of chunk ch + 1 are
            // loaded in iteration ch (independent loads; nothing waits for them in this iteration)
            int kp_n = c_begin < c_end ? kpad_op[chunk_op[c_begin]] : 0;
            int op_n = c_begin + 1 < c_end ? chunk_op[c_begin + 1] : 0;
            for (int ch = c_begin; ch < c_end; ++ch, ++j) {
                const int s = j % nst, a = j & 1;
                const uint32_t ph = (uint32_t)(j / nst) & 1u;
                const int kp = kp_n;
                kp_n = ch + 1 < c_end ? kpad_op[op_n] : 0;
                op_n = ch + 2 < c_end ? chunk_op[ch + 2] : 0;
                if (!mbar_wait_ab(smem_addr(&full[s]), ph, ab) || !mbar_wait_ab(smem_addr(&opf[s]), ph, ab) ||
                    (j >= 2 && !mbar_wait_ab(smem_addr(&acce[a]), (uint32_t)((j >> 1) - 1) & 1u, ab))) {
                    give_up(1);
                    break;
                }
                tc_after_sync();
                fence_async_smem();   // with the producers' fences: their copies are seen by the MMAs
                const uint32_t a0 = smem_addr(base + s * stage_bytes), b0 = a0 + 3 * A_PART;
                // descriptors of the first core matrices; the address field (bits 0-13, address /
                // 16) of a later K step, part or row block is reached by adding its offset / 16
                const uint64_t dA = smem_desc_sw128(a0), dB = smem_desc(b0, b_lbo, 128);
                const uint64_t t3 = (uint64_t)((2 * npad * 16) >> 4);   // row 2 npad: part 3
                const uint32_t d = tmem + (uint32_t)(a * 4 * npad);
                for (int ks = 0; ks < kp / 16; ++ks) {
                    const uint64_t ka = (uint64_t)((ks * 32) >> 4);   // 16 columns = 32 bytes
                    const uint64_t kb = (uint64_t)((ks * 2 * b_lbo) >> 4);
                    const uint64_t x1 = dA + ka, x2 = dA + ka + (uint64_t)(A_PART >> 4),
                                   x3 = dA + ka + (uint64_t)((2 * A_PART) >> 4);
                    const uint32_t acc = ks != 0;
                    mma_bf16(d, x1, dB + kb, id2, acc);                                // X1 [T1; T2]
                    mma_bf16(d + (uint32_t)(2 * npad), x2, dB + kb, id2, acc);         // X2 [T1; T2]
                    mma_bf16(d + (uint32_t)(3 * npad), x1, dB + kb + t3, id1, 1);      // X1 T3
                    mma_bf16(d + (uint32_t)(3 * npad), x3, dB + kb, id1, 1);           // X3 T1
                }
                mma_commit(smem_addr(&empty[s]));   // the stage may be refilled once these complete
                mma_commit(smem_addr(&accf[a]));    // the products are in accumulator set a
            }
            // every MMA issued by this CTA has completed before the tensor memory is freed
            mma_commit(smem_addr(&fin));
            mbar_wait(smem_addr(&fin), 0);
        }
        __syncwarp();
    } else {
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (tasks), column octets
        //      h, h + 4, ... (h = w / 4) ----
        const int q4 = warp & 3, h = warp >> 2;
        const int m = 32 * q4 + lane;
        const int ld = stage_ld(R);
        int j = 0;
        for (int ch = c_begin; ch < c_end; ++ch, ++j) {
            const int a = j & 1;
            const int t0 = chunk_t0[ch], nt = chunk_t0[ch + 1] - t0;
            const bool mine = mbar_wait_ab(smem_addr(&accf[a]), (uint32_t)(j >> 1) & 1u, ab);
            if (!bar_and(mine, 1, EPI_THREADS)) {   // all epilogue warps leave together
                if (threadIdx.x == 0) give_up(2);
                break;
            }
            tc_after_sync();
            const uint32_t trow = tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(a * 4 * npad);
            for (int cc = 8 * h; cc < npad; cc += 16) {
                uint32_t r[4][8];
#pragma unroll
                for (int blk = 0; blk < 4; ++blk)
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
                        : "=r"(r[blk][0]), "=r"(r[blk][1]), "=r"(r[blk][2]), "=r"(r[blk][3]), "=r"(r[blk][4]),
                          "=r"(r[blk][5]), "=r"(r[blk][6]), "=r"(r[blk][7])
                        : "r"(trow + (uint32_t)(blk * npad + cc)));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int u = 0; u < 8; ++u)   // X1 T1 + ((X1 T2 + X2 T1) + (X2 T2 + X1 T3 + X3 T1))
                    if (cc + u < R)
                        tile[m * ld + cc + u] =
                            __uint_as_float(r[0][u]) +
                            ((__uint_as_float(r[1][u]) + __uint_as_float(r[2][u])) + __uint_as_float(r[3][u]));
            }
            tc_before_sync();
            mbar_arrive(smem_addr(&acce[a]));   // accumulator set a may be overwritten
            bar_named(1, EPI_THREADS);           // the tile is complete
            write_products<TD, EPI_THREADS>(tile, ld, R, t0, nt, temp, task_dst, accumulate, dst, threadIdx.x);
            bar_named(1, EPI_THREADS);           // the tile may be refilled
        }
    }
    tc_before_sync();
    __syncthreads();
    if (warp == MMA_WARP) {
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

// Three-part bfloat16 image of one R x C operator (row-major, binary64) for the MMAs: out
// receives 3 * npad * kpad bfloat16 values (16-bit patterns), one image of 3 npad rows in the
// no-swizzle K-major layout of the file comment: part 1 (the value rounded to bfloat16 through
// binary32) in rows 0..npad-1, part 2 (the remainder, formed in binary64 and rounded) in rows
// npad..2 npad-1, part 3 (what is left, rounded) in rows 2 npad..3 npad-1.
void tc_operator_image(const double* op, int R, int C, int npad, int kpad, uint16_t* out) {
    std::memset(out, 0, 3 * (size_t)npad * kpad * sizeof(uint16_t));
    for (int r = 0; r < R; ++r)
        for (int k = 0; k < C; ++k) {
            const double a = op[(size_t)r * C + k];
            float b0, b1, b2;
            const uint16_t p0 = host_bf16((float)a, &b0);
            const uint16_t p1 = host_bf16((float)(a - (double)b0), &b1);
            const uint16_t p2 = host_bf16((float)(a - (double)b0 - (double)b1), &b2);
            out[img_off(r, k, 3 * npad) / 2] = p0;
            out[img_off(npad + r, k, 3 * npad) / 2] = p1;
            out[img_off(2 * npad + r, k, 3 * npad) / 2] = p2;
        }
}

// Shared memory of a launch: nst stages (source images of 128 rows and the operator image,
// three parts each, kmax columns), the product tile (128 x stage_ld(R) binary32) and 1 KB for
// the alignment of the base.
static size_t tc_smem_bytes(int nst, int npad, int kmax, int R) {
    return (size_t)nst * tc_stage_size(npad, kmax) + (size_t)TC_M * stage_ld(R) * 4 + 1024;
}

namespace {
struct TcDevice {
    bool ready = false;
    size_t cap = 0;   // dynamic shared memory a CTA may use
    int sms = 0;
};
TcDevice g_tc_dev[64];
}  // namespace

mh_status tc_prepare(mh_ctx* ctx) {
    if (ctx->device < 0 || ctx->device >= 64) return mh_fail(ctx, MH_ERR_INVALID_ARG, "device index out of range");
    TcDevice& d = g_tc_dev[ctx->device];
    if (d.ready) return MH_OK;
    int optin = 0, sms = 0;
    MH_CUDA(ctx, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    MH_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    cudaFuncAttributes fa{};
    MH_CUDA(ctx, cudaFuncGetAttributes(&fa, k_contract_tc<float>));
    const size_t cap = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
    // the largest operator (64 x 64) must fit two stages
    if (cap < tc_smem_bytes(2, 64, 64, 64))
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "device shared memory (%d B per block) too small for the tensor-core "
                       "contraction (%zu B)", optin, tc_smem_bytes(2, 64, 64, 64) + fa.sharedSizeBytes);
    MH_CUDA(ctx, cudaFuncSetAttribute(k_contract_tc<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap));
    MH_CUDA(ctx, cudaFuncSetAttribute(k_contract_tc<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap));
    d.cap = cap;
    d.sms = sms;
    d.ready = true;
    return MH_OK;
}

mh_status tc_contract_launch(mh_ctx* ctx, const tc_launch& a) {
    if (a.n_chunks == 0) return MH_OK;
    MH_TRY(tc_prepare(ctx));
    const TcDevice& d = g_tc_dev[ctx->device];
    if (a.npad > 64 || a.kmax > 64 || a.R > a.npad)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "tensor-core contraction too large (%d x %d)", a.npad, a.kmax);
    int nst = TC_MAX_STAGES;
    while (nst > 2 && tc_smem_bytes(nst, a.npad, a.kmax, a.R) > d.cap) --nst;
    const size_t smem = tc_smem_bytes(nst, a.npad, a.kmax, a.R);
    if (smem > d.cap) return mh_fail(ctx, MH_ERR_INVALID_ARG, "tensor-core contraction needs %zu B of shared memory", smem);
    const unsigned grid = (unsigned)std::min<int64_t>(a.n_chunks, d.sms);
    if (a.dst_double)
        k_contract_tc<double><<<grid, TC_THREADS, smem, ctx->stream>>>(
            reinterpret_cast<const __nv_bfloat16*>(a.img), a.img_off, a.kpad, a.chunk_op, a.chunk_t0,
            (int)a.n_chunks, a.spl, a.plane, a.tc_src, a.R, a.npad, a.kmax, nst, a.temp, a.task_dst, a.accumulate,
            static_cast<double*>(a.dst), a.err);
    else
        k_contract_tc<float><<<grid, TC_THREADS, smem, ctx->stream>>>(
            reinterpret_cast<const __nv_bfloat16*>(a.img), a.img_off, a.kpad, a.chunk_op, a.chunk_t0,
            (int)a.n_chunks, a.spl, a.plane, a.tc_src, a.R, a.npad, a.kmax, nst, a.temp, a.task_dst, a.accumulate,
            static_cast<float*>(a.dst), a.err);
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
