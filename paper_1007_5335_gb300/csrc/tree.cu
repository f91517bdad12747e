// Adaptive quadtree on the device (Section 3.1): level-by-level refinement of D by the
// interpolation-error predicate, 2:1 balancing, box numbering, leaf ordering and the
// adaptive multipole interaction lists U, V, W, X.
//
// Every level l keeps a dense status map of its 4^l cells indexed by Morton code
// (x bit below y bit): -1 absent, 1 leaf, 2 internal; after numbering the map holds
// box ids.  Neighbour lookups are therefore O(1) and no hashing is needed; for the
// supported depth (<= 10) all maps together take at most 1.4 M entries.
#include <algorithm>
#include <cmath>
#include <memory>

#include "mh_internal.cuh"

namespace {

constexpr int ST_ABSENT = -1, ST_LEAF = 1, ST_INTERNAL = 2;
constexpr int LIST_CAP = 32;

__host__ __device__ __forceinline__ uint32_t spread_bits(uint32_t v) {
    v &= 0x0000ffffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}
__host__ __device__ __forceinline__ uint32_t compact_bits(uint32_t v) {
    v &= 0x55555555u;
    v = (v | (v >> 1)) & 0x33333333u;
    v = (v | (v >> 2)) & 0x0f0f0f0fu;
    v = (v | (v >> 4)) & 0x00ff00ffu;
    v = (v | (v >> 8)) & 0x0000ffffu;
    return v;
}
__host__ __device__ __forceinline__ uint32_t morton(uint32_t ix, uint32_t iy) { return spread_bits(ix) | (spread_bits(iy) << 1); }

struct Maps {
    int32_t* st;        // concatenated per-level maps
    int64_t off[12];    // per level offset (level <= 10)
    int L;              // max level
};

__device__ __forceinline__ int32_t map_get(const Maps& M, int l, int ix, int iy) {
    const int n = 1 << l;
    if (l < 0 || ix < 0 || iy < 0 || ix >= n || iy >= n) return ST_ABSENT;
    return M.st[M.off[l] + morton(ix, iy)];
}

// ---- refinement ----

// Points at which the predicate needs F: per candidate box its own q*q nodes, then the
// q*q nodes of each child (child c = cx + 2 cy), node j = iy*q + ix.
__global__ void k_refine_points(const int32_t* __restrict__ cand, int64_t ncand, int l, double x0, double y0,
                                double W, const double* __restrict__ xi, int q, double* pts) {
    const int64_t i = blockIdx.x;
    if (i >= ncand) return;
    const uint32_t m = (uint32_t)cand[i];
    const int ix = (int)compact_bits(m), iy = (int)compact_bits(m >> 1);
    const double w = W / (double)(1 << l);
    const double cx = x0 + (ix + 0.5) * w, cy = y0 + (iy + 0.5) * w;
    const int qq = q * q;
    for (int e = threadIdx.x; e < 5 * qq; e += blockDim.x) {
        const int part = e / qq, j = e % qq;
        double bx = cx, by = cy, bw = w;
        if (part > 0) {
            const int c = part - 1;
            bw = 0.5 * w;
            bx = cx + ((c & 1) ? 0.25 : -0.25) * w;
            by = cy + ((c & 2) ? 0.25 : -0.25) * w;
        }
        double* p = pts + 2 * (i * 5 * qq + e);
        p[0] = bx + 0.5 * bw * xi[j % q];
        p[1] = by + 0.5 * bw * xi[j / q];
    }
}

// err = max over children nodes |F - P_b F|, P_b F the tensor interpolant on the box's
// own nodes; flag = err > tol.  Lc[s][i][a] = l_a(s/2 + xi_i/2), s = 0 (-) or 1 (+).
__global__ void k_refine_flag(const double* __restrict__ F, int64_t ncand, int q, const double* __restrict__ Lc,
                              double tol, int32_t* flag, double* err_out) {
    const int64_t i = blockIdx.x;
    if (i >= ncand) return;
    const int qq = q * q;
    const double* own = F + i * 5 * qq;
    double e = 0.0;
    for (int t = threadIdx.x; t < 4 * qq; t += blockDim.x) {
        const int c = t / qq, j = t % qq;
        const int nx = j % q, ny = j / q;
        const double* lx = Lc + ((c & 1) * q + nx) * q;
        const double* ly = Lc + (((c >> 1) & 1) * q + ny) * q;
        double acc = 0.0;
        for (int a = 0; a < q; ++a) {
            double row = 0.0;
            for (int b = 0; b < q; ++b) row += own[a * q + b] * lx[b];
            acc += ly[a] * row;
        }
        e = fmax(e, fabs(own[qq + t] - acc));
    }
    __shared__ double red[256];
    red[threadIdx.x] = e;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        flag[i] = red[0] > tol;
        err_out[i] = red[0];
    }
}

// Mark split boxes internal and create their children as leaves.
__global__ void k_apply_split(Maps M, int l, const int32_t* __restrict__ cand, const int32_t* __restrict__ flag,
                              int64_t ncand) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ncand || !flag[i]) return;
    const uint32_t m = (uint32_t)cand[i];
    M.st[M.off[l] + m] = ST_INTERNAL;
    for (int c = 0; c < 4; ++c) M.st[M.off[l + 1] + 4 * m + c] = ST_LEAF;
}

// Gather the cells of level l whose status equals `want` (cells in Morton order):
// per-block counts, then positions from an exclusive scan.
__global__ void k_count_status(const int32_t* __restrict__ st, int64_t n, int want, int32_t* bcount) {
    __shared__ int32_t cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && st[i] == want) atomicAdd(&cnt, 1);
    __syncthreads();
    if (threadIdx.x == 0) bcount[blockIdx.x] = cnt;
}

// Stable per-block compaction using a warp-ballot scan inside the block.
__global__ void k_gather_status(const int32_t* __restrict__ st, int64_t n, int want, const int32_t* __restrict__ boff,
                                int32_t* out) {
    __shared__ int32_t wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool hit = i < n && st[i] == want;
    const unsigned bal = __ballot_sync(0xffffffffu, hit);
    const int before = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    int base = 0;
    for (int w = 0; w < warp; ++w) base += wsum[w];
    if (hit) out[boff[blockIdx.x] + base + before] = (int32_t)i;
}

// ---- 2:1 balance ----

// A leaf must split when a neighbour at its level is internal and one of that
// neighbour's children touching the leaf is internal too.
__global__ void k_balance_flag(Maps M, int l, int32_t* flag, int* any) {
    const int64_t n = 1LL << (2 * l);
    int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= n) return;
    flag[m] = 0;
    if (M.st[M.off[l] + m] != ST_LEAF || l + 2 > M.L) return;
    const int ix = (int)compact_bits((uint32_t)m), iy = (int)compact_bits((uint32_t)m >> 1);
    bool need = false;
    for (int dy = -1; dy <= 1 && !need; ++dy)
        for (int dx = -1; dx <= 1 && !need; ++dx) {
            if (!dx && !dy) continue;
            const int nx = ix + dx, ny = iy + dy;
            if (map_get(M, l, nx, ny) != ST_INTERNAL) continue;
            for (int a = 0; a < 2; ++a)
                for (int c = 0; c < 2; ++c) {
                    if ((dx == 1 && a != 0) || (dx == -1 && a != 1)) continue;
                    if ((dy == 1 && c != 0) || (dy == -1 && c != 1)) continue;
                    if (map_get(M, l + 1, 2 * nx + a, 2 * ny + c) == ST_INTERNAL) need = true;
                }
        }
    if (need) {
        flag[m] = 1;
        *any = 1;
    }
}

__global__ void k_balance_apply(Maps M, int l, const int32_t* __restrict__ flag) {
    const int64_t n = 1LL << (2 * l);
    int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= n || !flag[m]) return;
    M.st[M.off[l] + m] = ST_INTERNAL;
    for (int c = 0; c < 4; ++c) M.st[M.off[l + 1] + 4 * m + c] = ST_LEAF;
}

// ---- numbering ----

__global__ void k_present(const int32_t* __restrict__ st, int64_t n, int32_t* f) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) f[i] = st[i] != ST_ABSENT;
}

// Single-pass block scan helpers (exclusive), used with a host loop over chunks.
// Inclusive scan of one value per thread over a block of 1024 threads: warp shuffles inside
// each warp, then the 32 warp sums scanned by the first warp.  wsum: 32 ints of shared memory;
// on return wsum[31] holds the block's sum.
__device__ __forceinline__ int32_t block_incl_scan_1024(int32_t v, int32_t* wsum) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int32_t w = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    return (warp ? wsum[warp - 1] : 0) + x;
}

// Exclusive scan of each 1024-entry block of `in` (out) and the block sums (bsum).
__global__ void __launch_bounds__(1024) k_block_scan(const int32_t* __restrict__ in, int64_t n, int32_t* out,
                                                     int32_t* bsum) {
    __shared__ int32_t wsum[32];
    const int64_t i = blockIdx.x * 1024LL + threadIdx.x;
    const int32_t v = i < n ? in[i] : 0;
    const int32_t incl = block_incl_scan_1024(v, wsum);
    if (i < n) out[i] = incl - v;
    if (threadIdx.x == 1023) bsum[blockIdx.x] = incl;
}

// Exclusive scan of n block counts by one block of 1024 threads (chunks of 1024 with a carry):
// off[i] = c[0] + ... + c[i - 1], *total = the sum of all.
__global__ void __launch_bounds__(1024) k_scan_offsets(const int32_t* __restrict__ c, int64_t n,
                                                       int32_t* __restrict__ off, int64_t* __restrict__ total) {
    __shared__ int32_t wsum[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const int32_t v = i < n ? c[i] : 0;
        const int32_t incl = block_incl_scan_1024(v, wsum);
        if (i < n) off[i] = (int32_t)(carry + incl - v);
        __syncthreads();   // every thread has read carry and wsum
        if (threadIdx.x == 1023) carry += incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_add_offsets(int32_t* out, int64_t n, const int32_t* __restrict__ boff) {
    int64_t i = blockIdx.x * 1024LL + threadIdx.x;
    if (i < n) out[i] += boff[blockIdx.x];
}

// box id = exclusive scan of presence over all levels (level-major, Morton within level)
__global__ void k_number_boxes(int32_t* st, const int32_t* __restrict__ ids, int64_t n, const int64_t* __restrict__ loff,
                               int L, int32_t* boxes, int32_t* is_leaf) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || st[i] == ST_ABSENT) return;
    int l = 0;
    while (l < L && i >= loff[l + 1]) ++l;
    const uint32_t m = (uint32_t)(i - loff[l]);
    const int id = ids[i];
    boxes[3 * id] = l;
    boxes[3 * id + 1] = (int)compact_bits(m);
    boxes[3 * id + 2] = (int)compact_bits(m >> 1);
    is_leaf[id] = st[i] == ST_LEAF;
    st[i] = id;
}

// Mark the first finest-level cell of every leaf (leaf order = Morton order of that cell).
__global__ void k_leaf_first_cell(const int32_t* __restrict__ boxes, const int32_t* __restrict__ is_leaf,
                                  int64_t nbox, int L, int32_t* fine) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nbox || !is_leaf[b]) return;
    const int l = boxes[3 * b];
    const uint32_t m = morton((uint32_t)boxes[3 * b + 1], (uint32_t)boxes[3 * b + 2]);
    fine[(int64_t)m << (2 * (L - l))] = 1;
}

__global__ void k_leaf_order(const int32_t* __restrict__ boxes, const int32_t* __restrict__ is_leaf, int64_t nbox,
                             int L, const int32_t* __restrict__ rank, int32_t* leaf_box, int32_t* box_leaf) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    if (!is_leaf[b]) {
        box_leaf[b] = -1;
        return;
    }
    const int l = boxes[3 * b];
    const uint32_t m = morton((uint32_t)boxes[3 * b + 1], (uint32_t)boxes[3 * b + 2]);
    const int r = rank[(int64_t)m << (2 * (L - l))];
    leaf_box[r] = (int32_t)b;
    box_leaf[b] = r;
}

__global__ void k_family(Maps M, const int32_t* __restrict__ boxes, int64_t nbox, int32_t* parent, int32_t* child) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    const int l = boxes[3 * b], ix = boxes[3 * b + 1], iy = boxes[3 * b + 2];
    parent[b] = l > 0 ? map_get(M, l - 1, ix >> 1, iy >> 1) : -1;
    for (int c = 0; c < 4; ++c)
        child[4 * b + c] = l < M.L ? map_get(M, l + 1, 2 * ix + (c & 1), 2 * iy + (c >> 1)) : -1;
}

__global__ void k_nodes(const int32_t* __restrict__ boxes, const int32_t* __restrict__ leaf_box, int64_t nleaf, int q,
                        double x0, double y0, double W, const double* __restrict__ xi, double* nodes) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int qq = q * q;
    if (e >= nleaf * qq) return;
    const int64_t i = e / qq;
    const int j = (int)(e % qq);
    const int b = leaf_box[i];
    const int l = boxes[3 * b];
    const double w = W / (double)(1 << l);
    nodes[2 * e] = x0 + (boxes[3 * b + 1] + 0.5) * w + 0.5 * w * xi[j % q];
    nodes[2 * e + 1] = y0 + (boxes[3 * b + 2] + 0.5) * w + 0.5 * w * xi[j / q];
}

// ---- lists ----

__device__ __forceinline__ void push_unique(int32_t* lst, int& n, int32_t v) {
    for (int i = 0; i < n; ++i)
        if (lst[i] == v) return;
    if (n < LIST_CAP) lst[n++] = v;
}

__device__ __forceinline__ bool is_leaf_id(const int32_t* box_leaf, int32_t id) { return id >= 0 && box_leaf[id] >= 0; }

// which: 0 U (leaves), 1 V (level >= 2), 2 W (leaves), 3 X (all boxes)
__global__ void k_lists(Maps M, const int32_t* __restrict__ boxes, const int32_t* __restrict__ box_leaf, int64_t nbox,
                        int which, int32_t* tmp, int32_t* cnt) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    const int l = boxes[3 * b], ix = boxes[3 * b + 1], iy = boxes[3 * b + 2];
    int32_t lst[LIST_CAP];
    int n = 0;
    const bool leaf = box_leaf[b] >= 0;
    if (which == 0 && leaf) {
        push_unique(lst, n, (int32_t)b);
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (!dx && !dy) continue;
                const int nx = ix + dx, ny = iy + dy, nside = 1 << l;
                if (nx < 0 || ny < 0 || nx >= nside || ny >= nside) continue;
                const int32_t id = map_get(M, l, nx, ny);
                if (id >= 0) {
                    if (is_leaf_id(box_leaf, id)) {
                        push_unique(lst, n, id);
                    } else {
                        for (int a = 0; a < 2; ++a)
                            for (int c = 0; c < 2; ++c) {
                                if ((dx == 1 && a) || (dx == -1 && !a) || (dy == 1 && c) || (dy == -1 && !c)) continue;
                                const int32_t ch = map_get(M, l + 1, 2 * nx + a, 2 * ny + c);
                                if (is_leaf_id(box_leaf, ch)) push_unique(lst, n, ch);
                            }
                    }
                } else {
                    const int32_t pid = map_get(M, l - 1, nx >> 1, ny >> 1);
                    if (is_leaf_id(box_leaf, pid)) push_unique(lst, n, pid);
                }
            }
    } else if (which == 1 && l >= 2) {
        const int px = ix >> 1, py = iy >> 1;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int32_t nb = map_get(M, l - 1, px + dx, py + dy);
                if (nb < 0 || is_leaf_id(box_leaf, nb)) continue;
                for (int c = 0; c < 4; ++c) {
                    const int cx = 2 * (px + dx) + (c & 1), cy = 2 * (py + dy) + (c >> 1);
                    if (abs(cx - ix) <= 1 && abs(cy - iy) <= 1) continue;
                    const int32_t id = map_get(M, l, cx, cy);
                    if (id >= 0) push_unique(lst, n, id);
                }
            }
    } else if (which == 2 && leaf) {
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (!dx && !dy) continue;
                const int32_t nb = map_get(M, l, ix + dx, iy + dy);
                if (nb < 0 || is_leaf_id(box_leaf, nb)) continue;
                for (int c = 0; c < 4; ++c) {
                    const int cx = 2 * (ix + dx) + (c & 1), cy = 2 * (iy + dy) + (c >> 1);
                    if (cx >= 2 * ix - 1 && cx <= 2 * ix + 2 && cy >= 2 * iy - 1 && cy <= 2 * iy + 2) continue;
                    const int32_t id = map_get(M, l + 1, cx, cy);
                    if (id >= 0) push_unique(lst, n, id);
                }
            }
    } else if (which == 3 && l >= 1) {
        const int px = ix >> 1, py = iy >> 1;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (!dx && !dy) continue;
                const int32_t nb = map_get(M, l - 1, px + dx, py + dy);
                if (!is_leaf_id(box_leaf, nb)) continue;
                const int cx = px + dx, cy = py + dy;
                if (ix >= 2 * cx - 1 && ix <= 2 * cx + 2 && iy >= 2 * cy - 1 && iy <= 2 * cy + 2) continue;
                push_unique(lst, n, nb);
            }
    }
    // insertion sort by box id
    for (int i = 1; i < n; ++i) {
        int32_t v = lst[i];
        int j = i - 1;
        while (j >= 0 && lst[j] > v) {
            lst[j + 1] = lst[j];
            --j;
        }
        lst[j + 1] = v;
    }
    for (int i = 0; i < n; ++i) tmp[b * LIST_CAP + i] = lst[i];
    cnt[b] = n;
}

__global__ void k_list_compact(const int32_t* __restrict__ tmp, const int32_t* __restrict__ cnt,
                               const int32_t* __restrict__ off, int64_t nbox, int32_t* items) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    for (int i = 0; i < cnt[b]; ++i) items[off[b] + i] = tmp[b * LIST_CAP + i];
}

// ---- interpolation helpers used by the volume and step code ----

__global__ void k_locate(Maps M, const int32_t* __restrict__ box_leaf, double x0, double y0, double W,
                         const double* __restrict__ xy, int64_t n, int32_t* leaf) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double px = xy[2 * i], py = xy[2 * i + 1];
    int32_t res = -1;
    for (int l = 0; l <= M.L; ++l) {
        const int ns = 1 << l;
        int ix = (int)floor((px - x0) / W * ns), iy = (int)floor((py - y0) / W * ns);
        ix = ix < 0 ? 0 : (ix >= ns ? ns - 1 : ix);
        iy = iy < 0 ? 0 : (iy >= ns ? ns - 1 : iy);
        const int32_t id = map_get(M, l, ix, iy);
        if (id < 0) break;
        if (box_leaf[id] >= 0) {
            res = box_leaf[id];
            break;
        }
    }
    leaf[i] = res;
}

// Leaf interpolant at n points: tensor Lagrange basis on the leaf's q x q Gauss-Legendre nodes
// in barycentric form l_a(s) = bw_a prod_{m != a} (s - xi_m) (bw_a = 1 / prod_{m != a}
// (xi_a - xi_m), precomputed), the products by prefix and suffix sweeps: no division on the
// slow binary64 pipe.
template <int Q>
__global__ void k_interp(const int32_t* __restrict__ boxes, const int32_t* __restrict__ leaf_box, double x0, double y0,
                         double W, const double* __restrict__ xi, const double* __restrict__ bw,
                         const double* __restrict__ vals, const double* __restrict__ xy, const int32_t* __restrict__ leaf,
                         int64_t n, double* out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int lf = leaf[i];
    const int b = leaf_box[lf];
    const int l = boxes[3 * b];
    const double w = W / (double)(1 << l);
    const double cx = x0 + (boxes[3 * b + 1] + 0.5) * w, cy = y0 + (boxes[3 * b + 2] + 0.5) * w;
    const double sx = (xy[2 * i] - cx) * (2.0 / w), sy = (xy[2 * i + 1] - cy) * (2.0 / w);
    double dxv[Q], dyv[Q], lx[Q], ly[Q];
#pragma unroll
    for (int m = 0; m < Q; ++m) {
        dxv[m] = sx - xi[m];
        dyv[m] = sy - xi[m];
    }
    double px = 1.0, py = 1.0;   // prefix products
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        lx[a] = px;
        ly[a] = py;
        px *= dxv[a];
        py *= dyv[a];
    }
    px = 1.0;
    py = 1.0;                    // suffix products
#pragma unroll
    for (int a = Q - 1; a >= 0; --a) {
        lx[a] *= px * bw[a];
        ly[a] *= py * bw[a];
        px *= dxv[a];
        py *= dyv[a];
    }
    const double* v = vals + (int64_t)lf * Q * Q;
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        double row = 0.0;
#pragma unroll
        for (int c = 0; c < Q; ++c) row = fma(v[a * Q + c], lx[c], row);
        acc = fma(ly[a], row, acc);
    }
    out[i] = acc;
}

struct TreeExtra {
    Maps maps;
    dbuf<double> xi, bw;   // Gauss-Legendre nodes on [-1, 1] and their barycentric weights
};

}  // namespace

// Gauss-Legendre nodes on [-1, 1] (increasing) and weights, Newton on the Legendre
// three-term recurrence (host, binary64).
void mh_gauss_legendre(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double z = cos(MH_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            double pn = n == 1 ? z : p1, pm = n == 1 ? 1.0 : p0;
            double dp = n * (z * pn - pm) / (z * z - 1.0);
            double dz = pn / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        double pn = n == 1 ? z : p1, pm = n == 1 ? 1.0 : p0;
        double dp = n * (z * pn - pm) / (z * z - 1.0);
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// exclusive scan of n int32 (device) into out, on the device; the total comes back to the host
// (it sizes what the caller allocates next)
static mh_status scan_i32(mh_ctx* ctx, const int32_t* in, int64_t n, int32_t* out, int64_t* total) {
    cudaStream_t st = ctx->stream;
    const int64_t nb = (n + 1023) / 1024;
    *total = 0;
    if (n == 0) return MH_OK;
    dbuf<int32_t> bsum, boff;
    dbuf<int64_t> dtot;
    MH_ALLOC(ctx, bsum, nb);
    MH_ALLOC(ctx, boff, nb);
    MH_ALLOC(ctx, dtot, 1);
    k_block_scan<<<(unsigned)nb, 1024, 0, st>>>(in, n, out, bsum.p);
    MH_LAUNCHED(ctx);
    k_scan_offsets<<<1, 1024, 0, st>>>(bsum.p, nb, boff.p, dtot.p);
    MH_LAUNCHED(ctx);
    k_add_offsets<<<(unsigned)nb, 1024, 0, st>>>(out, n, boff.p);
    MH_LAUNCHED(ctx);
    MH_CUDA(ctx, cudaMemcpyAsync(total, dtot.p, 8, cudaMemcpyDeviceToHost, st));
    MH_CUDA(ctx, cudaStreamSynchronize(st));
    return MH_OK;
}

// indices of the cells of one level map with status `want`, in Morton order
static mh_status gather_level(mh_ctx* ctx, const int32_t* st_level, int64_t n, int want, dbuf<int32_t>& out,
                              int64_t* count) {
    cudaStream_t s = ctx->stream;
    const int64_t nb = (n + 255) / 256;
    dbuf<int32_t> bc, bo;
    MH_ALLOC(ctx, bc, nb);
    MH_ALLOC(ctx, bo, nb);
    k_count_status<<<(unsigned)nb, 256, 0, s>>>(st_level, n, want, bc.p);
    MH_LAUNCHED(ctx);
    // block offsets on the device; only the count comes back (it sizes `out`)
    dbuf<int64_t> dtot;
    MH_ALLOC(ctx, dtot, 1);
    k_scan_offsets<<<1, 1024, 0, s>>>(bc.p, nb, bo.p, dtot.p);
    MH_LAUNCHED(ctx);
    int64_t acc = 0;
    MH_CUDA(ctx, cudaMemcpyAsync(&acc, dtot.p, 8, cudaMemcpyDeviceToHost, s));
    MH_CUDA(ctx, cudaStreamSynchronize(s));
    MH_ALLOC(ctx, out, std::max<int64_t>(acc, 1));
    k_gather_status<<<(unsigned)nb, 256, 0, s>>>(st_level, n, want, bo.p, out.p);
    MH_LAUNCHED(ctx);
    *count = acc;
    return MH_OK;
}

// Per-tree data private to this file (level maps, Gauss-Legendre nodes).
struct TreeWithExtra : mh_tree {
    TreeExtra ex;
};

static TreeExtra* extra_of(const mh_tree* t) { return &static_cast<TreeWithExtra*>(const_cast<mh_tree*>(t))->ex; }

extern "C" mh_status mh_tree_build(mh_ctx* ctx, const double* box3_host, int q, int min_level, int max_level,
                                   mh_field_fn refine_fn, void* user, double refine_tol, mh_tree** out) {
    if (!ctx || !box3_host || !out) return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (q < 2 || q > 16) return mh_fail(ctx, MH_ERR_INVALID_ARG, "q must be in 2..16");
    if (min_level < 0 || max_level < min_level || max_level > 10)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "need 0 <= min_level <= max_level <= 10");
    if (!(box3_host[2] > 0)) return mh_fail(ctx, MH_ERR_INVALID_ARG, "box width must be positive");
    cudaStream_t st = ctx->stream;
    auto* t = new TreeWithExtra();
    std::unique_ptr<TreeWithExtra> guard(t);
    for (int i = 0; i < 3; ++i) t->box[i] = box3_host[i];
    t->q = q;
    t->min_level = min_level;
    t->max_level = max_level;
    const int L = max_level;
    TreeExtra& E = t->ex;
    t->status_off.resize(L + 2);
    int64_t tot = 0;
    for (int l = 0; l <= L; ++l) {
        t->status_off[l] = tot;
        E.maps.off[l] = tot;
        tot += 1LL << (2 * l);
    }
    t->status_off[L + 1] = tot;
    E.maps.off[L + 1] = tot;
    E.maps.L = L;
    MH_ALLOC(ctx, t->status, tot);
    E.maps.st = t->status.p;
    MH_CUDA(ctx, cudaMemsetAsync(t->status.p, 0xff, tot * 4, st));   // -1 = absent
    const int32_t one = ST_LEAF;
    MH_CUDA(ctx, cudaMemcpyAsync(t->status.p, &one, 4, cudaMemcpyHostToDevice, st));
    // Gauss-Legendre nodes and the child interpolation matrices of the predicate
    std::vector<double> xi(q), wq(q), Lc(2 * q * q);
    mh_gauss_legendre(q, xi.data(), wq.data());
    for (int s = 0; s < 2; ++s)
        for (int i = 0; i < q; ++i) {
            double pt = (s ? 0.5 : -0.5) + 0.5 * xi[i];
            for (int a = 0; a < q; ++a) {
                double v = 1.0;
                for (int m = 0; m < q; ++m)
                    if (m != a) v *= (pt - xi[m]) / (xi[a] - xi[m]);
                Lc[(s * q + i) * q + a] = v;
            }
        }
    MH_ALLOC(ctx, E.xi, q);
    MH_ALLOC(ctx, E.bw, q);
    dbuf<double> dLc;
    MH_ALLOC(ctx, dLc, 2 * q * q);
    MH_CUDA(ctx, cudaMemcpyAsync(E.xi.p, xi.data(), q * 8, cudaMemcpyHostToDevice, st));
    {
        std::vector<double> bwh(q);
        for (int a = 0; a < q; ++a) {
            double d = 1.0;
            for (int m = 0; m < q; ++m)
                if (m != a) d *= xi[a] - xi[m];
            bwh[a] = 1.0 / d;
        }
        MH_CUDA(ctx, cudaMemcpyAsync(E.bw.p, bwh.data(), q * 8, cudaMemcpyHostToDevice, st));
        MH_CUDA(ctx, cudaStreamSynchronize(st));
    }
    MH_CUDA(ctx, cudaMemcpyAsync(dLc.p, Lc.data(), 2 * q * q * 8, cudaMemcpyHostToDevice, st));
    const int qq = q * q;
    // refinement, level by level
    for (int l = 0; l < L; ++l) {
        dbuf<int32_t> cand, flag;
        int64_t nc = 0;
        MH_TRY(gather_level(ctx, t->status.p + t->status_off[l], 1LL << (2 * l), ST_LEAF, cand, &nc));
        if (nc == 0) break;
        MH_ALLOC(ctx, flag, nc);
        if (l < min_level) {
            std::vector<int32_t> ones(nc, 1);
            MH_CUDA(ctx, cudaMemcpyAsync(flag.p, ones.data(), nc * 4, cudaMemcpyHostToDevice, st));
            MH_CUDA(ctx, cudaStreamSynchronize(st));
        } else if (refine_fn && std::isfinite(refine_tol)) {
            dbuf<double> pts, F, err;
            MH_ALLOC(ctx, pts, 2 * nc * 5 * qq);
            MH_ALLOC(ctx, F, nc * 5 * qq);
            MH_ALLOC(ctx, err, nc);
            k_refine_points<<<(unsigned)nc, 128, 0, st>>>(cand.p, nc, l, t->box[0], t->box[1], t->box[2], E.xi.p, q,
                                                          pts.p);
            MH_LAUNCHED(ctx);
            std::vector<double> hp(2 * nc * 5 * qq), hf(nc * 5 * qq);
            MH_CUDA(ctx, cudaMemcpyAsync(hp.data(), pts.p, hp.size() * 8, cudaMemcpyDeviceToHost, st));
            MH_CUDA(ctx, cudaStreamSynchronize(st));
            if (refine_fn(hp.data(), nc * 5 * qq, hf.data(), user) != 0)
                return mh_fail(ctx, MH_ERR_CALLBACK, "refine_fn returned an error at level %d", l);
            MH_CUDA(ctx, cudaMemcpyAsync(F.p, hf.data(), hf.size() * 8, cudaMemcpyHostToDevice, st));
            k_refine_flag<<<(unsigned)nc, 256, 0, st>>>(F.p, nc, q, dLc.p, refine_tol, flag.p, err.p);
            MH_LAUNCHED(ctx);
        } else {
            MH_CUDA(ctx, cudaMemsetAsync(flag.p, 0, nc * 4, st));
        }
        k_apply_split<<<mh_grid(nc, 256), 256, 0, st>>>(E.maps, l, cand.p, flag.p, nc);
        MH_LAUNCHED(ctx);
    }
    // 2:1 balance
    {
        dbuf<int32_t> bflag;
        dbuf<int> any;
        MH_ALLOC(ctx, bflag, 1LL << (2 * L));
        MH_ALLOC(ctx, any, 1);
        for (int iter = 0; iter < 4 * (L + 1); ++iter) {
            MH_CUDA(ctx, cudaMemsetAsync(any.p, 0, 4, st));
            int h_any = 0;
            // finest levels first so that a split propagates coarser within one sweep
            for (int l = L - 2; l >= 0; --l) {
                const int64_t n = 1LL << (2 * l);
                k_balance_flag<<<mh_grid(n, 256), 256, 0, st>>>(E.maps, l, bflag.p, any.p);
                MH_LAUNCHED(ctx);
                k_balance_apply<<<mh_grid(n, 256), 256, 0, st>>>(E.maps, l, bflag.p);
                MH_LAUNCHED(ctx);
            }
            MH_CUDA(ctx, cudaMemcpyAsync(&h_any, any.p, 4, cudaMemcpyDeviceToHost, st));
            MH_CUDA(ctx, cudaStreamSynchronize(st));
            if (!h_any) break;
        }
    }
    // numbering: box ids by (level, Morton); leaves by Morton key of their first finest cell
    {
        dbuf<int32_t> pres, ids;
        MH_ALLOC(ctx, pres, tot);
        MH_ALLOC(ctx, ids, tot);
        k_present<<<mh_grid(tot, 256), 256, 0, st>>>(t->status.p, tot, pres.p);
        MH_LAUNCHED(ctx);
        int64_t nbox = 0;
        MH_TRY(scan_i32(ctx, pres.p, tot, ids.p, &nbox));
        t->n_boxes = nbox;
        dbuf<int64_t> loff;
        MH_ALLOC(ctx, loff, L + 2);
        MH_CUDA(ctx, cudaMemcpyAsync(loff.p, t->status_off.data(), (L + 2) * 8, cudaMemcpyHostToDevice, st));
        dbuf<int32_t> is_leaf;
        MH_ALLOC(ctx, t->boxes, 3 * nbox);
        MH_ALLOC(ctx, is_leaf, nbox);
        k_number_boxes<<<mh_grid(tot, 256), 256, 0, st>>>(t->status.p, ids.p, tot, loff.p, L, t->boxes.p, is_leaf.p);
        MH_LAUNCHED(ctx);
        const int64_t nfine = 1LL << (2 * L);
        dbuf<int32_t> fine, rank;
        MH_ALLOC(ctx, fine, nfine);
        MH_ALLOC(ctx, rank, nfine);
        MH_CUDA(ctx, cudaMemsetAsync(fine.p, 0, nfine * 4, st));
        k_leaf_first_cell<<<mh_grid(nbox, 256), 256, 0, st>>>(t->boxes.p, is_leaf.p, nbox, L, fine.p);
        MH_LAUNCHED(ctx);
        int64_t nleaf = 0;
        MH_TRY(scan_i32(ctx, fine.p, nfine, rank.p, &nleaf));
        t->n_leaves = nleaf;
        t->n_nodes = nleaf * qq;
        MH_ALLOC(ctx, t->leaf_box, nleaf);
        MH_ALLOC(ctx, t->box_leaf, nbox);
        k_leaf_order<<<mh_grid(nbox, 256), 256, 0, st>>>(t->boxes.p, is_leaf.p, nbox, L, rank.p, t->leaf_box.p,
                                                          t->box_leaf.p);
        MH_LAUNCHED(ctx);
        MH_ALLOC(ctx, t->box_parent, nbox);
        MH_ALLOC(ctx, t->box_child, 4 * nbox);
        k_family<<<mh_grid(nbox, 256), 256, 0, st>>>(E.maps, t->boxes.p, nbox, t->box_parent.p, t->box_child.p);
        MH_LAUNCHED(ctx);
        MH_ALLOC(ctx, t->nodes, 2 * t->n_nodes);
        k_nodes<<<mh_grid(t->n_nodes, 256), 256, 0, st>>>(t->boxes.p, t->leaf_box.p, nleaf, q, t->box[0], t->box[1],
                                                          t->box[2], E.xi.p, t->nodes.p);
        MH_LAUNCHED(ctx);
        // level ranges of box ids
        std::vector<int32_t> hb(3 * nbox);
        MH_CUDA(ctx, cudaMemcpyAsync(hb.data(), t->boxes.p, hb.size() * 4, cudaMemcpyDeviceToHost, st));
        MH_CUDA(ctx, cudaStreamSynchronize(st));
        t->lvl_start.assign(L + 2, (int32_t)nbox);
        for (int64_t b = nbox - 1; b >= 0; --b) t->lvl_start[hb[3 * b]] = (int32_t)b;
        for (int l = L; l >= 0; --l)
            if (t->lvl_start[l] > t->lvl_start[l + 1]) t->lvl_start[l] = t->lvl_start[l + 1];
    }
    // interaction lists
    t->list_len.assign(4, 0);
    {
        const int64_t nbox = t->n_boxes;
        dbuf<int32_t> tmp, cnt;
        MH_ALLOC(ctx, tmp, nbox * LIST_CAP);
        MH_ALLOC(ctx, cnt, nbox);
        for (int w = 0; w < 4; ++w) {
            k_lists<<<mh_grid(nbox, 128), 128, 0, st>>>(E.maps, t->boxes.p, t->box_leaf.p, nbox, w, tmp.p, cnt.p);
            MH_LAUNCHED(ctx);
            MH_ALLOC(ctx, t->list_off[w], nbox + 1);
            int64_t total = 0;
            MH_TRY(scan_i32(ctx, cnt.p, nbox, t->list_off[w].p, &total));
            int32_t tt = (int32_t)total;
            MH_CUDA(ctx, cudaMemcpyAsync(t->list_off[w].p + nbox, &tt, 4, cudaMemcpyHostToDevice, st));
            MH_ALLOC(ctx, t->list_item[w], std::max<int64_t>(total, 1));
            k_list_compact<<<mh_grid(nbox, 256), 256, 0, st>>>(tmp.p, cnt.p, t->list_off[w].p, nbox,
                                                               t->list_item[w].p);
            MH_LAUNCHED(ctx);
            t->list_len[w] = total;
        }
    }
    MH_CUDA(ctx, cudaStreamSynchronize(st));
    *out = guard.release();
    return MH_OK;
}

extern "C" mh_status mh_tree_destroy(mh_tree* t) {
    if (t) {
        volume_free(t);
        delete static_cast<TreeWithExtra*>(t);
    }
    return MH_OK;
}

extern "C" mh_status mh_tree_size(const mh_tree* t, int64_t* nl, int64_t* nb, int64_t* nn) {
    if (!t) return MH_ERR_INVALID_ARG;
    if (nl) *nl = t->n_leaves;
    if (nb) *nb = t->n_boxes;
    if (nn) *nn = t->n_nodes;
    return MH_OK;
}

extern "C" mh_status mh_tree_boxes(mh_ctx* ctx, const mh_tree* t, int32_t* out_host) {
    if (!ctx || !t || !out_host) return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    MH_CUDA(ctx, cudaMemcpyAsync(out_host, t->boxes.p, 3 * t->n_boxes * 4, cudaMemcpyDeviceToHost, ctx->stream));
    MH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return MH_OK;
}

extern "C" mh_status mh_tree_leaves(mh_ctx* ctx, const mh_tree* t, int32_t* out_host) {
    if (!ctx || !t || !out_host) return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    std::vector<int32_t> lb(t->n_leaves), bx(3 * t->n_boxes);
    MH_CUDA(ctx, cudaMemcpyAsync(lb.data(), t->leaf_box.p, t->n_leaves * 4, cudaMemcpyDeviceToHost, ctx->stream));
    MH_CUDA(ctx, cudaMemcpyAsync(bx.data(), t->boxes.p, 3 * t->n_boxes * 4, cudaMemcpyDeviceToHost, ctx->stream));
    MH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int64_t i = 0; i < t->n_leaves; ++i)
        for (int c = 0; c < 3; ++c) out_host[3 * i + c] = bx[3 * lb[i] + c];
    return MH_OK;
}

extern "C" mh_status mh_tree_nodes(mh_ctx* ctx, const mh_tree* t, double* out_dev) {
    if (!ctx || !t || !out_dev) return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    MH_CUDA(ctx, cudaMemcpyAsync(out_dev, t->nodes.p, 2 * t->n_nodes * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    MH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return MH_OK;
}

extern "C" mh_status mh_tree_list(mh_ctx* ctx, const mh_tree* t, int which, int32_t* offsets_host, int32_t* items_host) {
    if (!ctx || !t || !offsets_host) return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    if (which < 0 || which > 3) return mh_fail(ctx, MH_ERR_INVALID_ARG, "which must be 0..3");
    MH_CUDA(ctx, cudaMemcpyAsync(offsets_host, t->list_off[which].p, (t->n_boxes + 1) * 4, cudaMemcpyDeviceToHost,
                                 ctx->stream));
    if (items_host && t->list_len[which] > 0)
        MH_CUDA(ctx, cudaMemcpyAsync(items_host, t->list_item[which].p, t->list_len[which] * 4,
                                     cudaMemcpyDeviceToHost, ctx->stream));
    MH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return MH_OK;
}

mh_status tree_locate(mh_ctx* ctx, const mh_tree* t, const double* xy_dev, int64_t n, int32_t* leaf_out) {
    if (n == 0) return MH_OK;
    k_locate<<<mh_grid(n, 256), 256, 0, ctx->stream>>>(extra_of(t)->maps, t->box_leaf.p, t->box[0], t->box[1],
                                                        t->box[2], xy_dev, n, leaf_out);
    MH_LAUNCHED(ctx);
    return MH_OK;
}

mh_status tree_interpolate(mh_ctx* ctx, const mh_tree* t, const double* vals, const double* xy_dev,
                           const int32_t* leaf, int64_t n, double* out) {
    if (n == 0) return MH_OK;
    const TreeExtra* E = extra_of(t);
#define MH_INTERP(QV)                                                                                     \
    k_interp<QV><<<mh_grid(n, 128), 128, 0, ctx->stream>>>(t->boxes.p, t->leaf_box.p, t->box[0], t->box[1],  \
                                                            t->box[2], E->xi.p, E->bw.p, vals, xy_dev, leaf, n, out)
    switch (t->q) {
        case 2: MH_INTERP(2); break;
        case 3: MH_INTERP(3); break;
        case 4: MH_INTERP(4); break;
        case 5: MH_INTERP(5); break;
        case 6: MH_INTERP(6); break;
        case 7: MH_INTERP(7); break;
        case 8: MH_INTERP(8); break;
        case 9: MH_INTERP(9); break;
        case 10: MH_INTERP(10); break;
        case 11: MH_INTERP(11); break;
        case 12: MH_INTERP(12); break;
        case 13: MH_INTERP(13); break;
        case 14: MH_INTERP(14); break;
        case 15: MH_INTERP(15); break;
        case 16: MH_INTERP(16); break;
        default: return mh_fail(ctx, MH_ERR_INVALID_ARG, "interpolation order q=%d not instantiated", t->q);
    }
#undef MH_INTERP
    MH_LAUNCHED(ctx);
    return MH_OK;
}

const double* tree_gl_nodes(const mh_tree* t) { return extra_of(t)->xi.p; }
