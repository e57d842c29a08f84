// build.cu -- LBVH construction for each rigid part of a mesh (once per mesh load).
//
//   1. Morton codes: 30-bit code of each triangle centroid, quantised in its
//      part's rest-pose bounding box, with the part's layout rank in bits
//      32..35 so one global sort keeps every part contiguous.
//   2. Stable LSD radix sort of (key, triangle) pairs, 8 bits per pass,
//      written from scratch (histogram, exclusive scan, warp-ordered scatter).
//   3. Binary radix tree of each part's sorted keys (Karras, "Maximizing
//      parallelism in the construction of BVHs, octrees, and k-d trees",
//      HPG 2012), duplicate keys split by position; children, parents.
//   4. Node depth, for the traversal stack bound.
#include "srp_internal.cuh"

namespace srp {

// spread the low 10 bits of v to every third bit
__device__ inline unsigned spread3(unsigned v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__global__ void k_morton(const double *rest64, const int *tri_vidx, const int *tri_part, const int *rank_of_part,
                         const int *tri_grp, const float *part_lo, const float *part_ext, int n_tris,
                         unsigned long long *keys, int *vals)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tris) return;
    int p = tri_part[t];
    float c[3];
    for (int k = 0; k < 3; k++) {
        double s = rest64[3 * tri_vidx[3 * t] + k] + rest64[3 * tri_vidx[3 * t + 1] + k] +
                   rest64[3 * tri_vidx[3 * t + 2] + k];
        c[k] = (float)(s / 3.0);
    }
    // one scale for all three axes (the part's largest extent): per-axis scaling
    // would give a thin axis as many code bits as a long one, and the radix tree
    // would split thin structures (a panel's frame) into overlapping halves
    const float e = fmaxf(fmaxf(part_ext[3 * p], part_ext[3 * p + 1]), part_ext[3 * p + 2]);
    unsigned q[3];
    for (int k = 0; k < 3; k++) {
        float f = e > 0.f ? (c[k] - part_lo[3 * p + k]) / e : 0.5f;
        f = fminf(fmaxf(f, 0.f), 1.f);
        q[k] = min((unsigned)(f * 1024.f), 1023u);
    }
    unsigned m = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
    // part rank, then coplanar group (0: none), then the Morton code: every group
    // of a part is one subtree of the part's radix tree
    keys[t] = ((unsigned long long)rank_of_part[p] << 48) | ((unsigned long long)(tri_grp[t] & 0xffff) << 32) | m;
    vals[t] = t;
}

cudaError_t launch_morton(const double *rest64, const int *tri_vidx, const int *tri_part, const int *rank_of_part,
                          const int *tri_grp, const float *part_lo, const float *part_ext, int n_tris,
                          unsigned long long *keys, int *vals, cudaStream_t st)
{
    k_morton<<<(n_tris + 255) / 256, 256, 0, st>>>(rest64, tri_vidx, tri_part, rank_of_part, tri_grp, part_lo,
                                                   part_ext, n_tris, keys, vals);
    return cudaGetLastError();
}

// ------------------------------------------------------------ radix sort
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;                       // per thread
constexpr int kSortTile = kSortThreads * kSortItems;  // elements per block
constexpr int kWarps = kSortThreads / 32;
constexpr int kPerWarp = kSortTile / kWarps;

size_t radix_sort_scratch_ints(int n)
{
    int nb = (n + kSortTile - 1) / kSortTile;
    return (size_t)256 * nb + 256;
}

__global__ void k_hist(const unsigned long long *keys, int n, int shift, int nb, int *hist)
{
    __shared__ int h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    int base = blockIdx.x * kSortTile;
    for (int i = threadIdx.x; i < kSortTile; i += blockDim.x) {
        int g = base + i;
        if (g < n) atomicAdd(&h[(keys[g] >> shift) & 0xff], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i * nb + blockIdx.x] = h[i];
}

// exclusive scan of m ints in place (single block of 1024 threads)
__global__ void k_scan(int *a, int m)
{
    __shared__ int part[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < m; base += 1024) {
        int i = base + threadIdx.x;
        int v = i < m ? a[i] : 0;
        part[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            int x = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
            __syncthreads();
            part[threadIdx.x] += x;
            __syncthreads();
        }
        int incl = part[threadIdx.x];
        if (i < m) a[i] = carry + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += incl;
        __syncthreads();
    }
}

// Stable scatter: warp w owns elements [w*kPerWarp, (w+1)*kPerWarp) of the
// block's tile; per-warp digit counts give each warp its starting offsets,
// then each warp walks its range in order, 32 at a time, ranking equal digits
// by lane with __match_any_sync.
__global__ void k_scatter(const unsigned long long *keys, const int *vals, unsigned long long *ko, int *vo, int n,
                          int shift, int nb, const int *hist)
{
    __shared__ int cnt[kWarps][256];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < kWarps * 256; i += blockDim.x) (&cnt[0][0])[i] = 0;
    __syncthreads();
    int base = blockIdx.x * kSortTile + warp * kPerWarp;
    for (int i = lane; i < kPerWarp; i += 32) {
        int g = base + i;
        if (g < n) atomicAdd(&cnt[warp][(keys[g] >> shift) & 0xff], 1);
    }
    __syncthreads();
    // thread d turns the counts of digit d into per-warp global offsets
    for (int d = threadIdx.x; d < 256; d += blockDim.x) {
        int off = hist[d * nb + blockIdx.x];
        for (int w = 0; w < kWarps; w++) {
            int c = cnt[w][d];
            cnt[w][d] = off;
            off += c;
        }
    }
    __syncthreads();
    unsigned lt = (1u << lane) - 1u;
    for (int i0 = 0; i0 < kPerWarp; i0 += 32) {
        int g = base + i0 + lane;
        bool ok = g < n;
        unsigned long long k = ok ? keys[g] : 0ull;
        int dig = ok ? (int)((k >> shift) & 0xff) : 256;
        unsigned same = __match_any_sync(0xffffffffu, dig);
        int rank = __popc(same & lt);
        if (ok) {
            int pos = cnt[warp][dig] + rank;
            ko[pos] = k;
            vo[pos] = vals[g];
        }
        __syncwarp();
        // highest lane of each digit group advances that digit's offset
        if (ok && (same >> lane) == 1u) cnt[warp][dig] += __popc(same);
        __syncwarp();
    }
}

cudaError_t radix_sort_pairs(unsigned long long *keys, int *vals, unsigned long long *keys_tmp, int *vals_tmp, int n,
                             int lo_bit, int hi_bit, int *scratch, size_t scratch_ints, cudaStream_t st)
{
    if (n <= 1) return cudaSuccess;
    int nb = (n + kSortTile - 1) / kSortTile;
    if (scratch_ints < radix_sort_scratch_ints(n)) return cudaErrorInvalidValue;
    unsigned long long *ka = keys, *kb = keys_tmp;
    int *va = vals, *vb = vals_tmp;
    int passes = 0;
    for (int shift = lo_bit; shift < hi_bit; shift += 8) {
        k_hist<<<nb, kSortThreads, 0, st>>>(ka, n, shift, nb, scratch);
        k_scan<<<1, 1024, 0, st>>>(scratch, 256 * nb);
        k_scatter<<<nb, kSortThreads, 0, st>>>(ka, va, kb, vb, n, shift, nb, scratch);
        unsigned long long *tk = ka; ka = kb; kb = tk;
        int *tv = va; va = vb; vb = tv;
        passes++;
    }
    if (passes & 1) {
        cudaMemcpyAsync(keys, ka, sizeof(unsigned long long) * n, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(vals, va, sizeof(int) * n, cudaMemcpyDeviceToDevice, st);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------ Karras tree
// common-prefix length of sorted keys i and j of one part (-1 out of range);
// equal keys are told apart by their positions
__device__ inline int delta(const unsigned long long *k, int n, int i, int j)
{
    if (j < 0 || j >= n) return -1;
    unsigned long long a = k[i], b = k[j];
    if (a != b) return __clzll(a ^ b);
    return 64 + __clz((unsigned)(i ^ j));
}

// Thread per internal node g (global index).  Part-local refs: child >= 0 is
// an internal node, child < 0 is leaf ~t (part-local sorted triangle).
__global__ void k_karras(const unsigned long long *keys, const int *part_tri_begin, const int *part_tri_count,
                         const int *part_node_begin, const int *node_part, int n_internal_total, int4 *node_refs,
                         int *leaf_parent)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_internal_total) return;
    int p = node_part[g];
    int n = part_tri_count[p];
    int i = g - part_node_begin[p];
    const unsigned long long *k = keys + part_tri_begin[p];
    int d = (delta(k, n, i, i + 1) - delta(k, n, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = delta(k, n, i, i - d);
    int lmax = 2;
    while (delta(k, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(k, n, i, i + (l + t) * d) > dmin) l += t;
    int j = i + l * d;
    int dnode = delta(k, n, i, j);
    // split: largest s in [0, l) with delta(i, i + s d) > dnode, by halving steps
    int s = 0;
    for (int div = 2;; div <<= 1) {
        int t = (l + div - 1) / div;
        if (delta(k, n, i, i + (s + t) * d) > dnode) s += t;
        if (t <= 1) break;
    }
    int gamma = i + s * d + (d < 0 ? d : 0);
    int lo = min(i, j), hi = max(i, j);
    int left = (lo == gamma) ? ~gamma : gamma;
    int right = (hi == gamma + 1) ? ~(gamma + 1) : gamma + 1;
    int4 r = node_refs[g];
    r.x = left;
    r.y = right;
    node_refs[g] = r;
    int nb = part_node_begin[p];
    int tb = part_tri_begin[p];
    if (left >= 0) node_refs[nb + left].z = i; else leaf_parent[tb + ~left] = i;
    if (right >= 0) node_refs[nb + right].z = i; else leaf_parent[tb + ~right] = i;
}

cudaError_t launch_karras(const unsigned long long *keys, const int *part_tri_begin, const int *part_tri_count,
                          const int *part_node_begin, int n_parts_layout, int n_internal_total, const int *node_part,
                          int4 *node_refs, int *leaf_parent, cudaStream_t st)
{
    (void)n_parts_layout;
    if (n_internal_total <= 0) return cudaSuccess;
    k_karras<<<(n_internal_total + 255) / 256, 256, 0, st>>>(keys, part_tri_begin, part_tri_count, part_node_begin,
                                                            node_part, n_internal_total, node_refs, leaf_parent);
    return cudaGetLastError();
}

// depth of every internal node (root = 0) by walking parent links
__global__ void k_depth(const int4 *node_refs, const int *node_part_base, int n_nodes, int *depth_max)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_nodes) return;
    int base = node_part_base[g];
    int dep = 0, cur = g - base;
    while (true) {
        int par = node_refs[base + cur].z;
        if (par < 0 || dep > 100000) break;
        cur = par;
        dep++;
    }
    atomicMax(depth_max, dep);
}

cudaError_t launch_depth(const int4 *node_refs, const int *node_part_base, int n_nodes, int *depth, cudaStream_t st)
{
    if (n_nodes <= 0) return cudaSuccess;
    k_depth<<<(n_nodes + 255) / 256, 256, 0, st>>>(node_refs, node_part_base, n_nodes, depth);
    return cudaGetLastError();
}

}  // namespace srp
