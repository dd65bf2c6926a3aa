// Occupancy-map front end: static segments and sampled points from a raster.
//
// The paper's crowds live on generated maps of traversable ground and static
// objects, with start and end points sampled on the traversable part (Sec.
// 3.1 "Hierarchical Urban Generation", Sec. 3.2 "Interactive Dynamics
// Generation").  Given such a map as a raster, these kernels produce the
// inputs of the crowd step:
//   - the free/obstacle boundary as maximal axis-aligned segments, each
//     directed with its free side on the left (one thread per boundary line
//     counts its runs, a scan places them, the same threads write them);
//   - points uniform over the cells that are free with a clearance of c
//     cells, drawn with Philox4x32-10 (counter = (point, stream, 0, 0),
//     key = seed), so that any point can be drawn independently and the
//     draws are reproducible on any device.
// Coordinates are x0 + i * cell with the product and the sum rounded
// separately (no FMA), so results are bit-reproducible.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

#include "../../include/crowd.h"
#include "crowd_internal.h"
#include "philox.cuh"

namespace crowd {

crowd_status api_fail(crowd_status st, const char* fmt, ...);

namespace {

constexpr int kMapThreads = 256;
constexpr int kScanThreads = 1024;

__device__ __forceinline__ bool free_at(const uint8_t* occ, int W, int H, int x, int y, int closed) {
    if (x < 0 || y < 0 || x >= W || y >= H) return !closed;
    return occ[(size_t)y * W + x] == 0;
}

__device__ __forceinline__ float coord(float o, int i, float h) { return __fadd_rn(o, __fmul_rn((float)i, h)); }

// Boundary line `line`: horizontal lines y = y0 + j h (j = line, 0..H), then
// vertical lines x = x0 + i h (i = line - H - 1, 0..W).  Without `out` the
// runs are counted into counts[line]; with it they are written from
// out[offsets[line]] on.
__global__ void __launch_bounds__(kMapThreads) map_lines(const uint8_t* occ, int W, int H, float h, float x0,
                                                         float y0, int closed, int* counts, const int* offsets,
                                                         float4* out) {
    const int line = blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= H + W + 2) return;
    int n = 0;
    const int base = out ? offsets[line] : 0;
    if (line <= H) {
        const int j = line;  // between row j - 1 (below) and row j (above)
        int x = 0;
        while (x < W) {
            const bool below = free_at(occ, W, H, x, j - 1, closed), above = free_at(occ, W, H, x, j, closed);
            if (below == above) {
                ++x;
                continue;
            }
            const bool side = above;
            const int xs = x;
            while (x < W && free_at(occ, W, H, x, j - 1, closed) != free_at(occ, W, H, x, j, closed) &&
                   free_at(occ, W, H, x, j, closed) == side)
                ++x;
            if (out) {
                const float ya = coord(y0, j, h), xa = coord(x0, xs, h), xb = coord(x0, x, h);
                out[base + n] = side ? make_float4(xa, ya, xb, ya) : make_float4(xb, ya, xa, ya);
            }
            ++n;
        }
    } else {
        const int i = line - H - 1;  // between column i - 1 (left) and column i (right)
        int y = 0;
        while (y < H) {
            const bool left = free_at(occ, W, H, i - 1, y, closed), right = free_at(occ, W, H, i, y, closed);
            if (left == right) {
                ++y;
                continue;
            }
            const bool side = left;
            const int ys = y;
            while (y < H && free_at(occ, W, H, i - 1, y, closed) != free_at(occ, W, H, i, y, closed) &&
                   free_at(occ, W, H, i - 1, y, closed) == side)
                ++y;
            if (out) {
                const float xa = coord(x0, i, h), ya = coord(y0, ys, h), yb = coord(y0, y, h);
                out[base + n] = side ? make_float4(xa, ya, xa, yb) : make_float4(xa, yb, xa, ya);
            }
            ++n;
        }
    }
    if (!out) counts[line] = n;
}

// Exclusive scan of in[0..n) into out[0..n], out[n] = total, by one block:
// each thread sums a contiguous chunk, the chunk sums are scanned in shared
// memory, each thread then writes its chunk.
__global__ void __launch_bounds__(kScanThreads) scan_one_block(const int* in, int* out, int n) {
    __shared__ long long part[kScanThreads];
    const int t = threadIdx.x;
    const int chunk = (n + kScanThreads - 1) / kScanThreads;
    const int lo = min(n, t * chunk), hi = min(n, lo + chunk);
    long long s = 0;
    for (int k = lo; k < hi; ++k) s += in[k];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < kScanThreads; o <<= 1) {
        const long long v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    long long run = part[t] - s;
    for (int k = lo; k < hi; ++k) {
        out[k] = (int)run;
        run += in[k];
    }
    if (t == kScanThreads - 1) out[n] = (int)part[t];
}

__device__ __forceinline__ bool eligible(const uint8_t* occ, int W, int H, int x, int y, int closed, int c) {
    for (int dy = -c; dy <= c; ++dy)
        for (int dx = -c; dx <= c; ++dx)
            if (!free_at(occ, W, H, x + dx, y + dy, closed)) return false;
    return true;
}

// One thread per row: count its eligible cells, or (with `list`) write their
// row-major indices from list[offsets[y]] on.
__global__ void __launch_bounds__(kMapThreads) map_rows(const uint8_t* occ, int W, int H, int closed, int c,
                                                        int* counts, const int* offsets, int* list) {
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= H) return;
    int n = 0;
    const int base = list ? offsets[y] : 0;
    for (int x = 0; x < W; ++x)
        if (eligible(occ, W, H, x, y, closed, c)) {
            if (list) list[base + n] = y * W + x;
            ++n;
        }
    if (!list) counts[y] = n;
}

__global__ void __launch_bounds__(kMapThreads) map_points(const int* list, int M, int W, float h, float x0,
                                                          float y0, uint2 key, uint32_t stream, int n,
                                                          float2* out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint4 u = philox4x32_10(make_uint4((uint32_t)k, stream, 0u, 0u), key);
    const int idx = (int)(((unsigned long long)u.x * (unsigned long long)M) >> 32);
    const int cell = list[idx];
    const int cx = cell % W, cy = cell / W;
    const float fx = (float)(u.y >> 8) * 0x1p-24f, fy = (float)(u.z >> 8) * 0x1p-24f;
    const float tx = __fadd_rn((float)cx, fx), ty = __fadd_rn((float)cy, fy);
    out[k] = make_float2(__fadd_rn(x0, __fmul_rn(tx, h)), __fadd_rn(y0, __fmul_rn(ty, h)));
}

crowd_status check_map(const uint8_t* occ, int32_t W, int32_t H, float cell, float x0, float y0) {
    if (W < 1 || H < 1 || W > (1 << 15) || H > (1 << 15))
        return api_fail(CROWD_EINVAL, "map size must be in [1, 32768] x [1, 32768]");
    if (!occ) return api_fail(CROWD_EINVAL, "occ is null");
    if (!(cell > 0.f) || !std::isfinite(cell) || !std::isfinite(x0) || !std::isfinite(y0))
        return api_fail(CROWD_EINVAL, "cell must be finite and > 0, x0 and y0 finite");
    return CROWD_OK;
}

struct Scratch {
    int* p = nullptr;
    ~Scratch() {
        if (p) cudaFree(p);
    }
};

crowd_status map_cuda_fail(cudaError_t e, const char* what) {
    return api_fail(e == cudaErrorMemoryAllocation ? CROWD_ENOMEM : CROWD_ECUDA, "%s: %s", what,
                    cudaGetErrorString(e));
}

}  // namespace
}  // namespace crowd

using namespace crowd;

extern "C" crowd_status crowd_map_segments(const uint8_t* occ, int32_t W, int32_t H, float cell, float x0, float y0,
                                           int32_t closed, int32_t max_segments, float* segments,
                                           int32_t* n_segments, void* stream) {
    if (!n_segments) return api_fail(CROWD_EINVAL, "n_segments is null");
    *n_segments = 0;
    crowd_status st = check_map(occ, W, H, cell, x0, y0);
    if (st) return st;
    if (max_segments < 0 || (max_segments > 0 && !segments))
        return api_fail(CROWD_EINVAL, "max_segments < 0, or segments null");
    cudaStream_t s = (cudaStream_t)stream;
    const int lines = H + W + 2;
    Scratch buf;  // counts [lines], offsets [lines + 1]
    cudaError_t e = cudaMalloc((void**)&buf.p, sizeof(int) * (2 * (size_t)lines + 1));
    if (e != cudaSuccess) return map_cuda_fail(e, "map scratch");
    int* counts = buf.p;
    int* offsets = buf.p + lines;
    const int blocks = (lines + kMapThreads - 1) / kMapThreads;
    map_lines<<<blocks, kMapThreads, 0, s>>>(occ, W, H, cell, x0, y0, closed ? 1 : 0, counts, nullptr, nullptr);
    scan_one_block<<<1, kScanThreads, 0, s>>>(counts, offsets, lines);
    int total = 0;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&total, offsets + lines, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return map_cuda_fail(e, "map segment count");
    *n_segments = total;
    if (total > max_segments)
        return api_fail(CROWD_EINVAL, "the map has %d boundary segments, more than max_segments = %d", total,
                        max_segments);
    if (total > 0) {
        map_lines<<<blocks, kMapThreads, 0, s>>>(occ, W, H, cell, x0, y0, closed ? 1 : 0, nullptr, offsets,
                                                 (float4*)segments);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return map_cuda_fail(e, "map segments");
    }
    return CROWD_OK;
}

extern "C" crowd_status crowd_map_sample(const uint8_t* occ, int32_t W, int32_t H, float cell, float x0, float y0,
                                         int32_t closed, int32_t clearance, uint64_t seed, uint32_t stream_id,
                                         int32_t n_points, float* points, int32_t* n_eligible, void* stream) {
    if (!n_eligible) return api_fail(CROWD_EINVAL, "n_eligible is null");
    *n_eligible = 0;
    crowd_status st = check_map(occ, W, H, cell, x0, y0);
    if (st) return st;
    if (clearance < 0 || clearance > CROWD_MAP_MAX_CLEARANCE)
        return api_fail(CROWD_EINVAL, "clearance must be in [0, %d] cells", CROWD_MAP_MAX_CLEARANCE);
    if (n_points < 0 || (n_points > 0 && !points)) return api_fail(CROWD_EINVAL, "n_points < 0, or points null");
    cudaStream_t s = (cudaStream_t)stream;
    Scratch buf;  // counts [H], offsets [H + 1], list [W * H]
    cudaError_t e = cudaMalloc((void**)&buf.p, sizeof(int) * (2 * (size_t)H + 1 + (size_t)W * H));
    if (e != cudaSuccess) return map_cuda_fail(e, "map scratch");
    int* counts = buf.p;
    int* offsets = buf.p + H;
    int* list = offsets + H + 1;
    const int blocks = (H + kMapThreads - 1) / kMapThreads;
    map_rows<<<blocks, kMapThreads, 0, s>>>(occ, W, H, closed ? 1 : 0, clearance, counts, nullptr, nullptr);
    scan_one_block<<<1, kScanThreads, 0, s>>>(counts, offsets, H);
    int M = 0;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&M, offsets + H, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return map_cuda_fail(e, "map eligible count");
    *n_eligible = M;
    if (n_points == 0) return CROWD_OK;
    if (M == 0) return api_fail(CROWD_EINVAL, "no cell is free with a clearance of %d cells", clearance);
    map_rows<<<blocks, kMapThreads, 0, s>>>(occ, W, H, closed ? 1 : 0, clearance, nullptr, offsets, list);
    const uint2 key = make_uint2((uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32));
    map_points<<<(n_points + kMapThreads - 1) / kMapThreads, kMapThreads, 0, s>>>(list, M, W, cell, x0, y0, key,
                                                                                stream_id, n_points,
                                                                                (float2*)points);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return map_cuda_fail(e, "map points");
    return CROWD_OK;
}
