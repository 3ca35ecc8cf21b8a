// dressi_texgather.cu -- deterministic texel gradients: the texel-space gather
// alternative to red.global atomics (Sec. 3.3.2: the gradients of the four texels a
// bilinear sample reads "should be summed up").
//
// The adjoint writes one record per (pixel, layer) into a slot fixed by the pixel:
// key = the global index of the sample's base texel (ix0, iy0), payload = dL/dA
// (RGB) and the bilinear fractions (fx, fy); slots without a texture gradient keep
// the key TG_NONE.  Then:
//   1. a stable LSD radix sort (8-bit digits) orders the (key, slot) pairs by base
//      texel; the first pass drops TG_NONE keys; equal keys keep slot order;
//   2. a table gives each base texel the first sorted position of its records (-1
//      for none);
//   3. one thread per texel sums, in a fixed order, the records of the four bases
//      whose bilinear footprint holds the texel (itself, its left, upper and
//      upper-left neighbours, with REPEAT wrap) with the matching weights.
// No floating-point atomics: the result is bitwise reproducible.
#include "dressi_core.cuh"
#include "dressi_launch.h"

#include <algorithm>

namespace dressi {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;                      // items per thread per block
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;    // items per block
constexpr int RS_BINS = 256;

// --- device-wide exclusive scan of n non-negative ints (in place), three kernels ---
// Sums saturate at INT_MAX (for non-negative terms min(a + b, INT_MAX) is still
// associative), so a total past 2^31 - 1 reads as INT_MAX instead of wrapping.
constexpr int SC_THREADS = 1024;
constexpr int SC_ITEMS = 4;
constexpr int SC_TILE = SC_THREADS * SC_ITEMS;

__device__ __forceinline__ int sat_add(int a, int b)
{
    return a > 0x7fffffff - b ? 0x7fffffff : a + b;
}

__device__ __forceinline__ int block_excl_scan(int v, int *warp_tot, int &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x = sat_add(x, y);
    }
    int ex = __shfl_up_sync(0xffffffffu, x, 1);   // exclusive within the warp
    if (lane == 0) ex = 0;
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w = sat_add(w, y);
        }
        if (lane < nw) warp_tot[lane] = w;
    }
    __syncthreads();
    total = warp_tot[nw - 1];
    const int r = sat_add(ex, warp > 0 ? warp_tot[warp - 1] : 0);
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SC_THREADS) k_scan_reduce(const int *a, int n, int *partial)
{
    __shared__ int wt[32];
    const int base = blockIdx.x * SC_TILE + threadIdx.x * SC_ITEMS;
    int s = 0;
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) s = sat_add(s, (base + j < n) ? a[base + j] : 0);
    int total;
    block_excl_scan(s, wt, total);
    if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

// exclusive scan of the partials in one block (nparts <= SC_TILE); partial[nparts] = total
__global__ void __launch_bounds__(SC_THREADS) k_scan_partials(int *partial, int nparts)
{
    __shared__ int wt[32];
    const int base = threadIdx.x * SC_ITEMS;
    int v[SC_ITEMS], s = 0;
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        v[j] = (base + j < nparts) ? partial[base + j] : 0;
        s = sat_add(s, v[j]);
    }
    int total;
    int run = block_excl_scan(s, wt, total);
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        if (base + j < nparts) partial[base + j] = run;
        run = sat_add(run, v[j]);
    }
    if (threadIdx.x == 0) partial[nparts] = total;
}

__global__ void __launch_bounds__(SC_THREADS) k_scan_down(int *a, int n, const int *partial)
{
    __shared__ int wt[32];
    const int base = blockIdx.x * SC_TILE + threadIdx.x * SC_ITEMS;
    int v[SC_ITEMS], s = 0;
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        v[j] = (base + j < n) ? a[base + j] : 0;
        s = sat_add(s, v[j]);
    }
    int total;
    int run = sat_add(block_excl_scan(s, wt, total), partial[blockIdx.x]);
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        if (base + j < n) a[base + j] = run;
        run = sat_add(run, v[j]);
    }
}

// --- stable LSD radix sort pass ---------------------------------------------------
// Items [0, n) of keys_in/vals_in (n read from *count when count != nullptr);
// vals_in == nullptr means val = item index.  hist is [RS_BINS][nblocks].
__device__ __forceinline__ int rs_count(const int *count, long long cap)
{
    return count ? *count : (int)cap;
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const unsigned *keys, const int *count, long long cap,
                                                        int shift, int *hist, int nblocks)
{
    __shared__ int h[RS_BINS];
    const int n = rs_count(count, cap);
    const long long base = (long long)blockIdx.x * RS_TILE;
    if (base >= n) {   // past the records (the passes after the first see only the kept ones)
        hist[threadIdx.x * nblocks + blockIdx.x] = 0;
        return;
    }
    h[threadIdx.x] = 0;
    __syncthreads();
    for (int j = 0; j < RS_ITEMS; ++j) {
        const long long i = base + j * RS_THREADS + threadIdx.x;
        if (i < n) {
            const unsigned k = keys[i];
            if (k != TG_NONE) atomicAdd(&h[(k >> shift) & 0xff], 1);
        }
    }
    __syncthreads();
    hist[threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const unsigned *keys_in, const int *vals_in,
                                                           const int *count, long long cap, int shift,
                                                           const int *offs, int nblocks, unsigned *keys_out,
                                                           int *vals_out)
{
    __shared__ int run[RS_BINS];                     // next free position of each digit
    __shared__ int wcnt[RS_THREADS / 32][RS_BINS];   // per-warp digit counts of a round
    const int n = rs_count(count, cap);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long base = (long long)blockIdx.x * RS_TILE;
    if (base >= n) return;   // a block past the records has nothing to place
    run[tid] = offs[tid * nblocks + blockIdx.x];
    for (int j = 0; j < RS_ITEMS; ++j) {
        const long long i = base + j * RS_THREADS + tid;
        unsigned k = TG_NONE;
        if (i < n) k = keys_in[i];
        const bool valid = k != TG_NONE;
        // a round without a kept record (most of the first pass's slots are empty) places
        // nothing; the test is a barrier, so the previous round's counts are read
        if (!__syncthreads_or(valid)) continue;
        for (int w = 0; w < RS_THREADS / 32; ++w) wcnt[w][tid] = 0;
        __syncthreads();
        const int d = valid ? (int)((k >> shift) & 0xff) : RS_BINS;   // RS_BINS: dropped
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        // turn the per-warp counts of digit `tid` into exclusive offsets within the round
        {
            int acc = 0;
            for (int w = 0; w < RS_THREADS / 32; ++w) {
                const int c = wcnt[w][tid];
                wcnt[w][tid] = acc;
                acc += c;
            }
            __syncthreads();
            if (valid) {
                const int pos = run[d] + wcnt[warp][d] + rank;
                keys_out[pos] = k;
                vals_out[pos] = vals_in ? vals_in[i] : (int)i;
            }
            __syncthreads();
            run[tid] += acc;
        }
        __syncthreads();
    }
}

// --- gather ------------------------------------------------------------------------
// first[key] = the first sorted position holding key (the table starts at -1)
__global__ void k_tg_first(const unsigned *keys, const int *count, int *first)
{
    const int n = *count;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned k = keys[i];
        if (i == 0 || keys[i - 1] != k) first[k] = i;
    }
}

__global__ void k_tex_gather(Globals g, const unsigned *keys, const int *vals, const int *count, const int *first)
{
    const MeshK &M = g.meshes[blockIdx.y];
    const long long n_tex = (long long)M.tex_w * M.tex_h;
    const int n = *count;
    const float4 *p0 = g.tg_pay0;
    const float *p1 = g.tg_pay1;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n_tex;
         q += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(q % M.tex_w), y = (int)(q / M.tex_w);
        const int xl = x == 0 ? M.tex_w - 1 : x - 1, yu = y == 0 ? M.tex_h - 1 : y - 1;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
        // bases whose bilinear footprint holds (x, y): (x, y) as corner 00, (x-1, y) as 10,
        // (x, y-1) as 01, (x-1, y-1) as 11 (REPEAT wrap)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int bx = (c & 1) ? xl : x, by = (c & 2) ? yu : y;
            // a texture of width or height 1 wraps a texel onto itself: the same base
            // then owns several corners of the footprint, all handled by its records
            const unsigned key = (unsigned)(M.tex_off + (long long)by * M.tex_w + bx);
            int i = first[key];
            for (; i >= 0 && i < n && keys[i] == key; ++i) {
                const int slot = vals[i];
                const float4 r = p0[slot];
                const float fx = r.w, fy = p1[slot];
                const float wx = (c & 1) ? fx : 1.f - fx, wy = (c & 2) ? fy : 1.f - fy;
                const float w = wx * wy;
                a0 = fmaf(w, r.x, a0);
                a1 = fmaf(w, r.y, a1);
                a2 = fmaf(w, r.z, a2);
            }
        }
        reinterpret_cast<float4 *>(g.gtex)[M.tex_off + q] = make_float4(a0, a1, a2, 0.f);
    }
}

// --- driver -------------------------------------------------------------------------
static int grid_of(long long n, int block, int cap)
{
    long long b = (n + block - 1) / block;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

// the whole scan in one block, SC_TILE items at a time with a running carry (short arrays:
// one launch instead of three); the total goes where the three-kernel scan leaves it
__global__ void __launch_bounds__(SC_THREADS) k_scan_single(int *a, int n, int *total_out)
{
    __shared__ int wt[32];
    int carry = 0;
    for (int c0 = 0; c0 < n; c0 += SC_TILE) {
        const int base = c0 + threadIdx.x * SC_ITEMS;
        int v[SC_ITEMS], s = 0;
#pragma unroll
        for (int j = 0; j < SC_ITEMS; ++j) {
            v[j] = (base + j < n) ? a[base + j] : 0;
            s = sat_add(s, v[j]);
        }
        int total;
        int run = sat_add(block_excl_scan(s, wt, total), carry);
#pragma unroll
        for (int j = 0; j < SC_ITEMS; ++j) {
            if (base + j < n) a[base + j] = run;
            run = sat_add(run, v[j]);
        }
        carry = sat_add(carry, total);
    }
    if (threadIdx.x == 0) *total_out = carry;
}

void launch_scan_inplace(int *a, int n, int *partial, cudaStream_t s)
{
    if (n <= 2 * SC_TILE) {
        // partial[number of SC_TILE parts] = total, as k_scan_partials leaves it
        k_scan_single<<<1, SC_THREADS, 0, s>>>(a, n, partial + (n + SC_TILE - 1) / SC_TILE);
        count_launch(1);
        return;
    }
    const int nparts = (n + SC_TILE - 1) / SC_TILE;
    k_scan_reduce<<<nparts, SC_THREADS, 0, s>>>(a, n, partial);
    k_scan_partials<<<1, SC_THREADS, 0, s>>>(partial, nparts);
    k_scan_down<<<nparts, SC_THREADS, 0, s>>>(a, n, partial);
    count_launch(3);
}

int scan_partials_needed(long long n) { return (int)((n + SC_TILE - 1) / SC_TILE) + 1; }

size_t texgather_scratch_bytes(long long slots, long long n_texels, size_t align)
{
    const long long nblocks = (slots + RS_TILE - 1) / RS_TILE;
    const long long hist = (long long)RS_BINS * nblocks;
    const long long parts = (hist + SC_TILE - 1) / SC_TILE + 1;
    auto up = [align](size_t x) { return (x + align - 1) / align * align; };
    return up(sizeof(unsigned) * slots) * 2 + up(sizeof(int) * slots) * 2 + up(sizeof(int) * hist) +
           up(sizeof(int) * parts) + up(sizeof(int) * 4) + up(sizeof(int) * std::max<long long>(n_texels, 1));
}

void launch_tex_gather(const Globals &g, long long slots, long long n_texels, int n_meshes, int max_texels,
                       char *scratch, size_t align, cudaStream_t s)
{
    auto up = [align](size_t x) { return (x + align - 1) / align * align; };
    const long long nblocks = (slots + RS_TILE - 1) / RS_TILE;
    const long long hist_n = (long long)RS_BINS * nblocks;
    char *p = scratch;
    unsigned *kA = reinterpret_cast<unsigned *>(p); p += up(sizeof(unsigned) * slots);
    unsigned *kB = reinterpret_cast<unsigned *>(p); p += up(sizeof(unsigned) * slots);
    int *vA = reinterpret_cast<int *>(p); p += up(sizeof(int) * slots);
    int *vB = reinterpret_cast<int *>(p); p += up(sizeof(int) * slots);
    int *hist = reinterpret_cast<int *>(p); p += up(sizeof(int) * hist_n);
    int *partial = reinterpret_cast<int *>(p); p += up(sizeof(int) * ((hist_n + SC_TILE - 1) / SC_TILE + 1));
    int *count = reinterpret_cast<int *>(p); p += up(sizeof(int) * 4);
    int *first = reinterpret_cast<int *>(p);
    const int nparts = (int)((hist_n + SC_TILE - 1) / SC_TILE);

    // digits needed for the largest key
    int passes = 1;
    while (passes < 4 && (1ull << (8 * passes)) <= (unsigned long long)g.n_texels_max_key) ++passes;

    const unsigned *kin = g.tg_keys;
    const int *vin = nullptr;
    const int *cnt = nullptr;
    unsigned *kout = kA;
    int *vout = vA;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        k_rs_hist<<<(int)nblocks, RS_THREADS, 0, s>>>(kin, cnt, slots, shift, hist, (int)nblocks);
        launch_scan_inplace(hist, (int)hist_n, partial, s);
        if (pass == 0) {
            // the number of kept (valid) records is the scan's total
            cudaMemcpyAsync(count, partial + nparts, sizeof(int), cudaMemcpyDeviceToDevice, s);
        }
        k_rs_scatter<<<(int)nblocks, RS_THREADS, 0, s>>>(kin, vin, cnt, slots, shift, hist, (int)nblocks, kout, vout);
        count_launch(2);
        cnt = count;
        kin = kout;
        vin = vout;
        kout = (kout == kA) ? kB : kA;
        vout = (vout == vA) ? vB : vA;
    }
    cudaMemsetAsync(first, 0xff, sizeof(int) * (size_t)std::max<long long>(n_texels, 1), s);
    k_tg_first<<<grid_of(slots, 256, 152 * 16), 256, 0, s>>>(kin, count, first);
    dim3 grid(grid_of(max_texels, 256, 4096), n_meshes);
    k_tex_gather<<<grid, 256, 0, s>>>(g, kin, vin, count, first);
    count_launch(2);
}

// ---------------------------------------------------------------------------
// inverse UV (Sec. 3.3.2, Alg. 1): each texel takes the dL/d(albedo) of the sample
// that wrote it last (the largest sample number, kept by atomicMax in the adjoint);
// the sample's dL/dA waits in its record slot.  Texels without a writer stay 0.
// ---------------------------------------------------------------------------
__global__ void k_inv_uv_apply(Globals g, long long n_texels)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n_texels;
         t += (long long)gridDim.x * blockDim.x) {
        const int s = g.inv_uv[t];
        if (s < 0) continue;
        const float4 a = g.tg_pay0[s];
        reinterpret_cast<float4 *>(g.gtex)[t] = make_float4(a.x, a.y, a.z, 0.f);
    }
}

void launch_inv_uv_apply(const Globals &g, long long n_texels, cudaStream_t s)
{
    const long long blocks = std::min<long long>((n_texels + 255) / 256, 152LL * 32);
    k_inv_uv_apply<<<(int)std::max<long long>(blocks, 1), 256, 0, s>>>(g, n_texels);
    count_launch(1);
}

}  // namespace dressi
