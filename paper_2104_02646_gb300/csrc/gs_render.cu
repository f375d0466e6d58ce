// Differentiable soft rasteriser: the rendering stage of Sec. 2
// ("Differentiable rendering engine") that turns the simulated surface into
// images so that a loss on pixels reaches the vertex positions.  SoftRas-style
// sigmoid edges give every (pixel, triangle) pair a coverage D; the
// silhouette is the probabilistic union 1 - prod(1 - D); colours are
// DIB-R-style barycentric interpolations of vertex colours, blended by a
// softmax over the perspective-correct depth against a background.  The
// paper gives no formulas; the reading (the same one the FP64 oracle states)
// is spelled out at gs_raster_create in include/gradsim.h.
//
// Kernels:
//   k_rs_setup    one thread per triangle: project the corners (pinhole),
//                 twice the signed area, the pixel box its coverage can reach;
//   k_rs_bin_*    one CTA per (64x64 super-tile, chunk of triangles): test
//                 the chunk's 8-byte boxes against the super-tile's 16 tiles,
//                 count per tile, scan the counts (tile-major, chunks in
//                 order), then write every tile's list of triangle ids in
//                 ascending order (block scans keep the order);
//   k_rs_forward  one CTA per 16x16 tile, one warp per 8x4 pixel block, one
//                 thread per pixel, no block barrier: each warp culls its
//                 tile's ordered list against its block 32 entries at a time
//                 (8-byte boxes, ballot), and every pixel accumulates the hits
//                 in triangle order (product of 1 - D, online depth
//                 softmax); if the lists overflowed their buffer, the warp
//                 scans every triangle instead;
//   k_rs_backward one warp per triangle: its lanes walk the triangle's pixel
//                 box, recompute the pair exactly as the forward did, and
//                 accumulate dL/d(corner u, v, z, colour); a fixed xor tree
//                 reduces the lanes;
//   k_rs_vertex   one thread per vertex: fixed-order sum over its triangle
//                 corners (CSR built on the host), then the pinhole Jacobian
//                 back to world positions.
// No floating-point atomics: images and gradients are bitwise reproducible.

#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "gs_runtime.h"

namespace {

using gs::Buf;

constexpr int kTile = 16;             // tile side (pixels); 256 threads per tile CTA
constexpr int kTileThreads = kTile * kTile;
constexpr int kSuper = 64;            // super-tile side (pixels): 4 x 4 tiles
constexpr int kSub = (kSuper / kTile) * (kSuper / kTile);
constexpr float kTau = 1.0e-5f;       // outside coverage below this is none
constexpr float kQmin = 1.0e-6f;      // 1 - coverage is kept >= kQmin

struct Cam {
    float R[9], t[3];
    float fx, fy, cx, cy, z_near, z_far;
    int W, H;
};

struct Spec {
    float sigma, inv_sigma, r2, gamma, inv_gamma, eps;
    float bg[3];
};

// projected triangle (80 B)
struct TriScr {
    float ax, ay, bx, by;
    float cx, cy, A2, valid;
    float za, zb, zc, pad;
    int x0, y0, x1, y1;  // pixel box its coverage can reach (inclusive); x1 < x0 when culled
    int ia, ib, ic, pad2;
};

// dL/d(projected corners): (u, v, z) of a, b, c and their colours
struct TriGrad {
    float g[18];
    float pad[2];
};

__device__ __forceinline__ float cross2(float px, float py, float qx, float qy) { return px * qy - py * qx; }

__device__ __forceinline__ void cam_point(const Cam& c, const float* x, float& X, float& Y, float& Z) {
    X = c.R[0] * x[0] + c.R[1] * x[1] + c.R[2] * x[2] + c.t[0];
    Y = c.R[3] * x[0] + c.R[4] * x[1] + c.R[5] * x[2] + c.t[1];
    Z = c.R[6] * x[0] + c.R[7] * x[1] + c.R[8] * x[2] + c.t[2];
}

__global__ void k_rs_setup(const float* __restrict__ x, const int* __restrict__ faces, int F, Cam cam, Spec sp,
                           TriScr* __restrict__ out, short4* __restrict__ boxes) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    TriScr T;
    const int id[3] = {faces[3 * f], faces[3 * f + 1], faces[3 * f + 2]};
    float u[3], v[3], z[3];
    bool ok = true;
    for (int k = 0; k < 3; ++k) {
        float X, Y, Z;
        cam_point(cam, x + 3 * (size_t)id[k], X, Y, Z);
        z[k] = Z;
        ok = ok && Z > cam.z_near;
        const float iZ = 1.0f / Z;
        u[k] = cam.fx * X * iZ + cam.cx;
        v[k] = cam.fy * Y * iZ + cam.cy;
    }
    T.ax = u[0]; T.ay = v[0]; T.bx = u[1]; T.by = v[1]; T.cx = u[2]; T.cy = v[2];
    T.A2 = cross2(u[1] - u[0], v[1] - v[0], u[2] - u[0], v[2] - v[0]);
    T.za = z[0]; T.zb = z[1]; T.zc = z[2];
    T.ia = id[0]; T.ib = id[1]; T.ic = id[2];
    T.pad = 0.f;
    T.pad2 = 0;
    ok = ok && fabsf(T.A2) > 1e-12f && isfinite(T.A2);
    T.valid = ok ? 1.f : 0.f;
    T.x0 = 0; T.y0 = 0; T.x1 = -1; T.y1 = -1;
    if (ok) {
        // pixel centres (i + 0.5) within r of the triangle's bounding box
        const float r = sqrtf(sp.r2);
        const float lo_u = fminf(u[0], fminf(u[1], u[2])) - r, hi_u = fmaxf(u[0], fmaxf(u[1], u[2])) + r;
        const float lo_v = fminf(v[0], fminf(v[1], v[2])) - r, hi_v = fmaxf(v[0], fmaxf(v[1], v[2])) + r;
        const float x0 = ceilf(lo_u - 0.5f), x1 = floorf(hi_u - 0.5f);
        const float y0 = ceilf(lo_v - 0.5f), y1 = floorf(hi_v - 0.5f);
        // clamp in float to [-1, size] before converting (a box far off
        // screen stays empty, x0 > x1, without an out-of-range conversion)
        const float W = (float)cam.W, H = (float)cam.H;
        T.x0 = (int)fminf(fmaxf(x0, 0.f), W);
        T.x1 = (int)fmaxf(fminf(x1, W - 1.f), -1.f);
        T.y0 = (int)fminf(fmaxf(y0, 0.f), H);
        T.y1 = (int)fmaxf(fminf(y1, H - 1.f), -1.f);
        if (T.x0 > T.x1 || T.y0 > T.y1) {
            T.x0 = 0; T.y0 = 0; T.x1 = -1; T.y1 = -1;
        }
    }
    out[f] = T;
    boxes[f] = make_short4((short)T.x0, (short)T.y0, (short)T.x1, (short)T.y1);
}

__device__ __forceinline__ bool box_hits(short4 b, int x0, int y0, int x1, int y1) {
    return b.z >= x0 && b.x <= x1 && b.w >= y0 && b.y <= y1;
}

// Binning rounds: 256 threads x kPer consecutive triangles, so a thread's
// triangles are contiguous and threads follow triangle order.
constexpr int kPer = 8;
constexpr int kRound = 256 * kPer;

// block-wide exclusive scan of one int per thread (thread order); returns the total
__device__ __forceinline__ int block_exclusive_scan(int v, int& excl, int* s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < 8; ++w) {
        before += w < warp ? s_warp[w] : 0;
        total += s_warp[w];
    }
    excl = before + inc - v;
    __syncthreads();
    return total;
}

// tile t (0..15, row-major) of super-tile (x0, y0)
__device__ __forceinline__ bool tile_hits(short4 b, int x0, int y0, int t) {
    const int tx = x0 + kTile * (t % (kSuper / kTile)), ty = y0 + kTile * (t / (kSuper / kTile));
    return box_hits(b, tx, ty, tx + kTile - 1, ty + kTile - 1);
}

// CTA (super-tile blockIdx.x, triangle chunk blockIdx.y): per tile of the
// super-tile, how many of the chunk's triangle boxes overlap it; counts are
// indexed ((super-tile * 16 + tile) * chunks + chunk)
__global__ void __launch_bounds__(256) k_rs_bin_count(const short4* __restrict__ boxes, int F, int chunk, int nsx,
                                                      int W, int H, int* __restrict__ counts) {
    __shared__ int s_warp[8];
    const int x0 = (blockIdx.x % nsx) * kSuper, y0 = (blockIdx.x / nsx) * kSuper;
    const int x1 = min(x0 + kSuper, W) - 1, y1 = min(y0 + kSuper, H) - 1;
    const int fb = blockIdx.y * chunk, fe = min(fb + chunk, F);
    int n[kSub];
#pragma unroll
    for (int t = 0; t < kSub; ++t) n[t] = 0;
    for (int f = fb + threadIdx.x; f < fe; f += 256) {
        const short4 b = boxes[f];
        if (!box_hits(b, x0, y0, x1, y1)) continue;
#pragma unroll
        for (int t = 0; t < kSub; ++t) n[t] += tile_hits(b, x0, y0, t) ? 1 : 0;
    }
#pragma unroll 1
    for (int t = 0; t < kSub; ++t) {
        int excl;
        const int total = block_exclusive_scan(n[t], excl, s_warp);
        if (threadIdx.x == 0) counts[(blockIdx.x * kSub + t) * gridDim.y + blockIdx.y] = total;
    }
}

// exclusive scan of the super-tile counts (one CTA, fixed order); flags an
// overflow of the list buffer
__global__ void __launch_bounds__(256) k_rs_bin_scan(const int* __restrict__ counts, int n, long long cap,
                                                     int* __restrict__ offsets, int* __restrict__ overflow) {
    __shared__ long long part[256];
    const int per = (n + 255) / 256;
    const int b = threadIdx.x * per, e = min(b + per, n);
    long long s = 0;
    for (int i = b; i < e; ++i) s += counts[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long run = 0;
        for (int t = 0; t < 256; ++t) {
            const long long v = part[t];
            part[t] = run;
            run += v;
        }
        *overflow = run > cap ? 1 : 0;
    }
    __syncthreads();
    long long run = part[threadIdx.x];
    for (int i = b; i < e; ++i) {
        offsets[i] = (int)(run < cap ? run : cap);
        run += counts[i];
    }
}

// every tile's list: the chunk's triangle ids overlapping it, ascending;
// a tile's chunks are adjacent, so its list is ascending as a whole
__global__ void __launch_bounds__(256) k_rs_bin_fill(const short4* __restrict__ boxes, int F, int chunk, int nsx,
                                                     int W, int H, const int* __restrict__ offsets,
                                                     const int* __restrict__ overflow, int* __restrict__ lists) {
    __shared__ int s_warp[8];
    // tiles hit in a round: OR of the threads' masks, rotating over three
    // words so that clearing the next one never races with a reader
    __shared__ unsigned s_any[3];
    if (*overflow) return;
    const int x0 = (blockIdx.x % nsx) * kSuper, y0 = (blockIdx.x / nsx) * kSuper;
    const int x1 = min(x0 + kSuper, W) - 1, y1 = min(y0 + kSuper, H) - 1;
    const int fb = blockIdx.y * chunk, fe = min(fb + chunk, F);
    if (threadIdx.x < 3) s_any[threadIdx.x] = 0u;
    __syncthreads();
    int written[kSub];
#pragma unroll
    for (int t = 0; t < kSub; ++t) written[t] = 0;
    int round = 0;
    for (int base = fb; base < fe; base += kRound, ++round) {
        const int f0 = base + threadIdx.x * kPer;
        unsigned hm[kPer];  // per candidate: bit t = overlaps tile t
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            hm[k] = 0;
            if (f0 + k < fe) {
                const short4 b = boxes[f0 + k];
                if (box_hits(b, x0, y0, x1, y1)) {
#pragma unroll
                    for (int t = 0; t < kSub; ++t) hm[k] |= tile_hits(b, x0, y0, t) ? (1u << t) : 0u;
                }
            }
        }
        unsigned mine = 0;
#pragma unroll
        for (int k = 0; k < kPer; ++k) mine |= hm[k];
        if (threadIdx.x == 0) s_any[(round + 1) % 3] = 0u;
        if (mine) atomicOr(&s_any[round % 3], mine);
        __syncthreads();
        const unsigned any = s_any[round % 3];
#pragma unroll 1
        for (int t = 0; t < kSub; ++t) {
            if (!((any >> t) & 1u)) continue;  // uniform: no thread hit tile t
            int c = 0;
#pragma unroll
            for (int k = 0; k < kPer; ++k) c += (hm[k] >> t) & 1u;
            int excl;
            const int total = block_exclusive_scan(c, excl, s_warp);
            int* o = lists + offsets[(blockIdx.x * kSub + t) * gridDim.y + blockIdx.y] + written[t] + excl;
#pragma unroll
            for (int k = 0; k < kPer; ++k)
                if ((hm[k] >> t) & 1u) *o++ = f0 + k;
            written[t] += total;
        }
    }
}

__device__ __forceinline__ float seg_d2(float px, float py, float ex, float ey, float fx, float fy, float& t,
                                        float& rx, float& ry) {
    const float dx = fx - ex, dy = fy - ey;
    const float dd = fmaxf(dx * dx + dy * dy, 1e-30f);
    t = fminf(fmaxf(((px - ex) * dx + (py - ey) * dy) / dd, 0.f), 1.f);
    rx = px - (ex + t * dx);
    ry = py - (ey + t * dy);
    return rx * rx + ry * ry;
}

// One (pixel, triangle) pair, as the forward and the backward both evaluate it.
struct Pair {
    bool cover, inside, clamped;
    float w[3];      // barycentric weights
    float wc[3];     // clamped, normalised
    float S;         // sum of the clamped weights
    float d2;        // squared distance to the boundary
    int edge;        // nearest edge (0: ab, 1: bc, 2: ca)
    float et, erx, ery;  // its parameter and residual p - closest point
    float q, D;      // 1 - coverage (clamped), coverage
    float iz, zp, zh;
    float C[3];
};

__device__ __forceinline__ void eval_pair(const TriScr& T, float px, float py, const Spec& sp, const Cam& cam,
                                          const float* __restrict__ col, Pair& P) {
    const float pax = T.ax - px, pay = T.ay - py, pbx = T.bx - px, pby = T.by - py, pcx = T.cx - px,
                pcy = T.cy - py;
    const float iA2 = 1.0f / T.A2;
    P.w[0] = cross2(pbx, pby, pcx, pcy) * iA2;
    P.w[1] = cross2(pcx, pcy, pax, pay) * iA2;
    P.w[2] = cross2(pax, pay, pbx, pby) * iA2;
    P.inside = P.w[0] >= 0.f && P.w[1] >= 0.f && P.w[2] >= 0.f;
    float t0, r0x, r0y, t1, r1x, r1y, t2, r2x, r2y;
    const float d0 = seg_d2(px, py, T.ax, T.ay, T.bx, T.by, t0, r0x, r0y);
    const float d1 = seg_d2(px, py, T.bx, T.by, T.cx, T.cy, t1, r1x, r1y);
    const float d2 = seg_d2(px, py, T.cx, T.cy, T.ax, T.ay, t2, r2x, r2y);
    P.edge = 0; P.d2 = d0; P.et = t0; P.erx = r0x; P.ery = r0y;
    if (d1 < P.d2) { P.edge = 1; P.d2 = d1; P.et = t1; P.erx = r1x; P.ery = r1y; }
    if (d2 < P.d2) { P.edge = 2; P.d2 = d2; P.et = t2; P.erx = r2x; P.ery = r2y; }
    P.cover = P.inside || P.d2 <= sp.r2;
    if (!P.cover) return;
    const float tv = (P.inside ? P.d2 : -P.d2) * sp.inv_sigma;
    const float q = 1.0f / (1.0f + expf(tv));  // sigmoid(-tv)
    P.clamped = !(q > kQmin);
    P.q = P.clamped ? kQmin : q;
    P.D = 1.0f - P.q;
    float wp[3];
    P.S = 0.f;
    for (int k = 0; k < 3; ++k) {
        wp[k] = P.w[k] > 0.f ? P.w[k] : 0.f;
        P.S += wp[k];
    }
    const float iS = 1.0f / fmaxf(P.S, 1e-30f);
    for (int k = 0; k < 3; ++k) P.wc[k] = wp[k] * iS;
    P.iz = P.wc[0] / T.za + P.wc[1] / T.zb + P.wc[2] / T.zc;
    P.zp = 1.0f / P.iz;
    P.zh = (cam.z_far - P.zp) / (cam.z_far - cam.z_near);
    const int ids[3] = {T.ia, T.ib, T.ic};
    for (int c = 0; c < 3; ++c) P.C[c] = 0.f;
    for (int k = 0; k < 3; ++k)
        for (int c = 0; c < 3; ++c) P.C[c] += P.wc[k] * col[3 * (size_t)ids[k] + c];
}

__global__ void __launch_bounds__(kTileThreads)
    k_rs_forward(const TriScr* __restrict__ tris, const short4* __restrict__ boxes, int F,
                 const int* __restrict__ counts, const int* __restrict__ offsets, const int* __restrict__ overflow,
                 const int* __restrict__ lists, int n_super_x, int nch, const float* __restrict__ col, Cam cam,
                 Spec sp, float4* __restrict__ image, float4* __restrict__ image_keep, float4* __restrict__ aux) {
    // warp w owns the 8 x 4 pixel block (w % 2, w / 2) of the 16 x 16 tile;
    // warps run independently (no block barrier)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tx0 = blockIdx.x * kTile, ty0 = blockIdx.y * kTile;
    const int bx0 = tx0 + 8 * (warp & 1), by0 = ty0 + 4 * (warp >> 1);
    const int bx1 = min(bx0 + 7, cam.W - 1), by1 = min(by0 + 3, cam.H - 1);
    if (bx0 > bx1 || by0 > by1) return;  // the block lies off a ragged edge
    const int px = bx0 + (lane & 7), py = by0 + (lane >> 3);
    const bool active = px < cam.W && py < cam.H;
    const float fx = px + 0.5f, fy = py + 0.5f;
    // the tile's ordered list, or every triangle after an overflow
    const int st = (ty0 / kSuper) * n_super_x + tx0 / kSuper;
    const int sub = ((ty0 % kSuper) / kTile) * (kSuper / kTile) + (tx0 % kSuper) / kTile;
    const bool all = *overflow != 0;
    const int first = (st * kSub + sub) * nch, last = first + nch - 1;
    const int n_cand = all ? F : offsets[last] + counts[last] - offsets[first];
    const int* cand = all ? nullptr : lists + offsets[first];
    // running union and softmax, starting from the background at depth eps
    float Pq = 1.f, m = sp.eps, Z = 1.f;
    float N[3] = {sp.bg[0], sp.bg[1], sp.bg[2]};
    for (int base = 0; base < n_cand; base += 32) {
        const int c = base + lane;
        int f = -1;
        bool h = false;
        if (c < n_cand) {
            f = all ? c : cand[c];
            h = box_hits(boxes[f], bx0, by0, bx1, by1);
        }
        unsigned bal = __ballot_sync(0xffffffffu, h);
        while (bal) {  // the hits in list order
            const int src = __ffs(bal) - 1;
            bal &= bal - 1;
            const int fk = __shfl_sync(0xffffffffu, f, src);
            const TriScr S = tris[fk];
            if (!active || px < S.x0 || px > S.x1 || py < S.y0 || py > S.y1) continue;
            Pair P;
            eval_pair(S, fx, fy, sp, cam, col, P);
            if (!P.cover) continue;
            Pq *= P.q;
            if (P.zh > m) {
                const float sc = expf((m - P.zh) * sp.inv_gamma);
                Z *= sc;
                for (int k = 0; k < 3; ++k) N[k] *= sc;
                m = P.zh;
            }
            const float wgt = P.D * expf((P.zh - m) * sp.inv_gamma);
            Z += wgt;
            for (int k = 0; k < 3; ++k) N[k] += wgt * P.C[k];
        }
    }
    if (active) {
        const float iZ = 1.0f / Z;
        const float4 o = make_float4(N[0] * iZ, N[1] * iZ, N[2] * iZ, 1.0f - Pq);
        const size_t pi = (size_t)py * cam.W + px;
        image[pi] = o;
        image_keep[pi] = o;
        aux[pi] = make_float4(Pq, m, Z, 0.f);
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// dL/d(projected corners, colours) of one triangle, one warp
__global__ void k_rs_backward(const TriScr* __restrict__ tris, int F, const float* __restrict__ col, Cam cam,
                              Spec sp, const float4* __restrict__ image, const float4* __restrict__ aux,
                              const float4* __restrict__ gimg, TriGrad* __restrict__ out) {
    const int f = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (f >= F) return;
    const TriScr T = tris[f];
    float g[18];
    for (int k = 0; k < 18; ++k) g[k] = 0.f;
    const int bw = T.x1 - T.x0 + 1, bh = T.y1 - T.y0 + 1;
    const int n = (bw > 0 && bh > 0) ? bw * bh : 0;
    const float* const cols[3] = {col + 3 * (size_t)T.ia, col + 3 * (size_t)T.ib, col + 3 * (size_t)T.ic};
    for (int k = lane; k < n; k += 32) {
        const int px = T.x0 + k % bw, py = T.y0 + k / bw;
        const float fx = px + 0.5f, fy = py + 0.5f;
        Pair P;
        eval_pair(T, fx, fy, sp, cam, col, P);
        if (!P.cover) continue;
        const size_t pi = (size_t)py * cam.W + px;
        const float4 I = image[pi], ax = aux[pi], gI = gimg[pi];
        const float Pq = ax.x, m = ax.y, Z = ax.z;
        // silhouette A = 1 - prod q
        float gq = -gI.w * (Pq / P.q);
        // colour softmax
        const float e = expf((P.zh - m) * sp.inv_gamma);
        const float wgt = P.D * e;
        const float gw = (gI.x * (P.C[0] - I.x) + gI.y * (P.C[1] - I.y) + gI.z * (P.C[2] - I.z)) / Z;
        const float gC[3] = {gI.x * wgt / Z, gI.y * wgt / Z, gI.z * wgt / Z};
        const float gD = gw * e;
        const float gzh = gw * wgt * sp.inv_gamma;
        gq -= gD;  // D = 1 - q
        // q = sigmoid(-t), t = +-d2/sigma (unless clamped)
        float gd2 = 0.f;
        if (!P.clamped) {
            const float gt = gq * (-P.q * P.D);
            gd2 = gt * (P.inside ? sp.inv_sigma : -sp.inv_sigma);
        }
        // d2 = |p - e0 - t (e1 - e0)|^2 on the nearest edge: d/de0 = -2 r (1 - t), d/de1 = -2 r t
        {
            const float sx = -2.f * P.erx * gd2, sy = -2.f * P.ery * gd2;
            const float s0x = sx * (1.f - P.et), s0y = sy * (1.f - P.et), s1x = sx * P.et, s1y = sy * P.et;
            if (P.edge == 0) {  // a -> b
                g[0] += s0x; g[1] += s0y; g[3] += s1x; g[4] += s1y;
            } else if (P.edge == 1) {  // b -> c
                g[3] += s0x; g[4] += s0y; g[6] += s1x; g[7] += s1y;
            } else {  // c -> a
                g[6] += s0x; g[7] += s0y; g[0] += s1x; g[1] += s1y;
            }
        }
        // zh -> zp -> iz
        const float gzp = -gzh / (cam.z_far - cam.z_near);
        const float giz = -gzp * P.zp * P.zp;
        const float zs[3] = {T.za, T.zb, T.zc};
        float gwc[3];
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) {
            const float cx = cols[kk][0], cy = cols[kk][1], cz = cols[kk][2];
            gwc[kk] = giz / zs[kk] + gC[0] * cx + gC[1] * cy + gC[2] * cz;
            g[3 * kk + 2] += -giz * P.wc[kk] / (zs[kk] * zs[kk]);
            g[9 + 3 * kk + 0] += gC[0] * P.wc[kk];
            g[9 + 3 * kk + 1] += gC[1] * P.wc[kk];
            g[9 + 3 * kk + 2] += gC[2] * P.wc[kk];
        }
        // wc = max(w, 0) / S
        const float dotw = gwc[0] * P.wc[0] + gwc[1] * P.wc[1] + gwc[2] * P.wc[2];
        const float iS = 1.0f / fmaxf(P.S, 1e-30f);
        float gwb[3];
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) gwb[kk] = P.w[kk] > 0.f ? (gwc[kk] - dotw) * iS : 0.f;
        // w_k = alpha_k / A2, A2 = cross(b - a, c - a)
        const float iA2 = 1.0f / T.A2;
        const float ga0 = gwb[0] * iA2, ga1 = gwb[1] * iA2, ga2 = gwb[2] * iA2;
        const float gA2 = -(gwb[0] * P.w[0] + gwb[1] * P.w[1] + gwb[2] * P.w[2]) * iA2;
        const float pax = T.ax - fx, pay = T.ay - fy, pbx = T.bx - fx, pby = T.by - fy, pcx = T.cx - fx,
                    pcy = T.cy - fy;
        // alpha_a = cross(pb, pc), alpha_b = cross(pc, pa), alpha_c = cross(pa, pb)
        g[3] += ga0 * pcy;  g[4] += -ga0 * pcx;  g[6] += -ga0 * pby; g[7] += ga0 * pbx;
        g[6] += ga1 * pay;  g[7] += -ga1 * pax;  g[0] += -ga1 * pcy; g[1] += ga1 * pcx;
        g[0] += ga2 * pby;  g[1] += -ga2 * pbx;  g[3] += -ga2 * pay; g[4] += ga2 * pax;
        const float e1x = T.bx - T.ax, e1y = T.by - T.ay, e2x = T.cx - T.ax, e2y = T.cy - T.ay;
        const float gbx = gA2 * e2y, gby = -gA2 * e2x, gcx = -gA2 * e1y, gcy = gA2 * e1x;
        g[3] += gbx; g[4] += gby; g[6] += gcx; g[7] += gcy;
        g[0] -= gbx + gcx; g[1] -= gby + gcy;
    }
    TriGrad G;
    for (int k = 0; k < 18; ++k) G.g[k] = warp_sum(g[k]);
    G.pad[0] = G.pad[1] = 0.f;
    if (lane == 0) out[f] = G;
}

// per vertex: fixed-order sum over its (triangle, corner) entries, then the
// pinhole Jacobian: u = fx X/Z + cx, v = fy Y/Z + cy, z = Z, (X, Y, Z) = R x + t
__global__ void k_rs_vertex(const int* __restrict__ rowptr, const int* __restrict__ entries,
                            const TriGrad* __restrict__ tg, const float* __restrict__ x, Cam cam, int N,
                            float* __restrict__ dx, float* __restrict__ dcol) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float gu = 0.f, gv = 0.f, gz = 0.f, gc[3] = {0.f, 0.f, 0.f};
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
        const int e = entries[k], f = e >> 2, c = e & 3;
        const float* G = tg[f].g;
        gu += G[3 * c];
        gv += G[3 * c + 1];
        gz += G[3 * c + 2];
        for (int j = 0; j < 3; ++j) gc[j] += G[9 + 3 * c + j];
    }
    if (dcol)
        for (int j = 0; j < 3; ++j) dcol[3 * (size_t)i + j] = gc[j];
    if (dx) {
        float X, Y, Z;
        cam_point(cam, x + 3 * (size_t)i, X, Y, Z);
        const float iZ = 1.0f / Z;
        const float gX = gu * cam.fx * iZ, gY = gv * cam.fy * iZ;
        const float gZ = gz - (gu * cam.fx * X + gv * cam.fy * Y) * iZ * iZ;
        for (int j = 0; j < 3; ++j) dx[3 * (size_t)i + j] = cam.R[j] * gX + cam.R[3 + j] * gY + cam.R[6 + j] * gZ;
    }
}

}  // namespace

struct gs_raster {
    gs_ctx* ctx = nullptr;
    int N = 0, F = 0;
    Cam cam{};
    Spec sp{};
    Buf faces, tri, tgrad, rowptr, entries, img, aux, x, col;
    Buf boxes, bin_counts, bin_offsets, bin_flag, bin_lists;
    int nsx = 0, nsy = 0, nch = 1, chunk = 1;
    long long bin_cap = 0;
    bool have_forward = false;
};

static gs_status check_camera(const gs_camera& c) {
    const float v[] = {c.R[0], c.R[1], c.R[2], c.R[3], c.R[4], c.R[5], c.R[6], c.R[7], c.R[8],
                       c.t[0], c.t[1], c.t[2], c.fx, c.fy, c.cx, c.cy, c.z_near, c.z_far};
    for (float a : v)
        if (!std::isfinite(a)) return gs::set_error(GS_EINVAL, "non-finite camera parameter");
    if (c.width <= 0 || c.height <= 0 || c.width > 16384 || c.height > 16384)
        return gs::set_error(GS_EINVAL, "image size must be in [1, 16384]");
    if (!(c.z_near > 0.f) || !(c.z_far > c.z_near)) return gs::set_error(GS_EINVAL, "need 0 < z_near < z_far");
    if (c.fx == 0.f || c.fy == 0.f) return gs::set_error(GS_EINVAL, "zero focal length");
    return GS_OK;
}

static void set_camera(gs_raster* r, const gs_camera& c) {
    for (int k = 0; k < 9; ++k) r->cam.R[k] = c.R[k];
    for (int k = 0; k < 3; ++k) r->cam.t[k] = c.t[k];
    r->cam.fx = c.fx;
    r->cam.fy = c.fy;
    r->cam.cx = c.cx;
    r->cam.cy = c.cy;
    r->cam.z_near = c.z_near;
    r->cam.z_far = c.z_far;
    r->cam.W = c.width;
    r->cam.H = c.height;
}

extern "C" gs_status gs_raster_create(gs_ctx* ctx, const gs_raster_desc* d, gs_raster** out) try {
    gs::clear_error();
    if (!ctx || !d || !out) return gs::set_error(GS_EINVAL, "null argument");
    *out = nullptr;
    if (d->n_vertices <= 0 || d->n_faces < 0 || (d->n_faces > 0 && !d->faces))
        return gs::set_error(GS_EINVAL, "need n_vertices > 0, n_faces >= 0 and faces");
    if (d->n_faces > (1 << 29)) return gs::set_error(GS_EINVAL, "too many faces");
    GS_TRY(check_camera(d->camera));
    const float sv[] = {d->sigma, d->gamma, d->eps, d->bg[0], d->bg[1], d->bg[2]};
    for (float a : sv)
        if (!std::isfinite(a)) return gs::set_error(GS_EINVAL, "non-finite raster parameter");
    if (!(d->sigma > 0.f) || !(d->gamma > 0.f)) return gs::set_error(GS_EINVAL, "sigma and gamma must be > 0");
    const int N = d->n_vertices, F = d->n_faces;
    std::vector<int> rowptr(N + 1, 0), entries(3 * (size_t)F);
    for (int f = 0; f < F; ++f) {
        for (int c = 0; c < 3; ++c) {
            const int v = d->faces[3 * f + c];
            if (v < 0 || v >= N) return gs::set_error(GS_EINVAL, "face index out of range");
            rowptr[v + 1]++;
        }
    }
    for (int i = 0; i < N; ++i) rowptr[i + 1] += rowptr[i];
    {
        std::vector<int> fill(rowptr.begin(), rowptr.end() - 1);
        for (int f = 0; f < F; ++f)
            for (int c = 0; c < 3; ++c) entries[fill[d->faces[3 * f + c]]++] = (f << 2) | c;  // ascending f
    }
    auto r = new gs_raster;
    r->ctx = ctx;
    r->N = N;
    r->F = F;
    set_camera(r, d->camera);
    r->sp.sigma = d->sigma;
    r->sp.inv_sigma = 1.0f / d->sigma;
    r->sp.r2 = (float)(d->sigma * std::log((1.0 - kTau) / kTau));
    r->sp.gamma = d->gamma;
    r->sp.inv_gamma = 1.0f / d->gamma;
    r->sp.eps = d->eps;
    for (int c = 0; c < 3; ++c) r->sp.bg[c] = d->bg[c];
    cudaStream_t s = nullptr;
    const size_t P = (size_t)r->cam.W * r->cam.H;
    gs_status st = GS_OK;
    auto up = [&](Buf& b, const void* src, size_t bytes) -> gs_status {
        GS_TRY(b.alloc(ctx, std::max<size_t>(bytes, 16), s));
        if (bytes) GS_CUDA(cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, s));
        return GS_OK;
    };
    if ((st = up(r->faces, d->faces, 12 * (size_t)F)) < 0 || (st = up(r->rowptr, rowptr.data(), 4 * (size_t)(N + 1))) < 0 ||
        (st = up(r->entries, entries.data(), 4 * entries.size())) < 0 ||
        (st = r->tri.alloc(ctx, std::max<size_t>(sizeof(TriScr) * F, 16), s)) < 0 ||
        (st = r->tgrad.alloc(ctx, std::max<size_t>(sizeof(TriGrad) * F, 16), s)) < 0 ||
        (st = r->img.alloc(ctx, 16 * P, s)) < 0 || (st = r->aux.alloc(ctx, 16 * P, s)) < 0 ||
        (st = r->x.alloc(ctx, 12 * (size_t)N, s)) < 0 || (st = r->col.alloc(ctx, 12 * (size_t)N, s)) < 0) {
        delete r;
        return st;
    }
    // tile lists: 8 entries per triangle (at least 1 M) before the tiles fall back to scanning every triangle
    r->nsx = (r->cam.W + kSuper - 1) / kSuper;
    r->nsy = (r->cam.H + kSuper - 1) / kSuper;
    r->bin_cap = std::max<long long>(8LL * F, 1 << 20);
    // triangle chunks per super-tile: about four CTAs per SM in the binning kernels
    const int n_super = r->nsx * r->nsy;
    r->nch = std::max(1, std::min(64, (4 * std::max(ctx->num_sms, 1)) / n_super));
    r->chunk = std::max(kRound, ((F + r->nch - 1) / r->nch + kRound - 1) / kRound * kRound);
    r->nch = std::max(1, (F + r->chunk - 1) / r->chunk);
    if ((st = r->boxes.alloc(ctx, std::max<size_t>(8 * (size_t)F, 16), s)) < 0 ||
        (st = r->bin_counts.alloc(ctx, 4 * (size_t)n_super * kSub * r->nch, s)) < 0 ||
        (st = r->bin_offsets.alloc(ctx, 4 * (size_t)n_super * kSub * r->nch, s)) < 0 ||
        (st = r->bin_flag.alloc(ctx, 16, s)) < 0 || (st = r->bin_lists.alloc(ctx, 4 * (size_t)r->bin_cap, s)) < 0) {
        delete r;
        return st;
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        delete r;
        return gs::cuda_error(e, "gs_raster_create");
    }
    *out = r;
    return GS_OK;
} GS_ABI_CATCH

extern "C" void gs_raster_destroy(gs_raster* r) {
    if (!r) return;
    cudaDeviceSynchronize();
    delete r;
}

extern "C" gs_status gs_raster_set_camera(gs_raster* r, const gs_camera* c) try {
    gs::clear_error();
    if (!r || !c) return gs::set_error(GS_EINVAL, "null argument");
    if (c->width != r->cam.W || c->height != r->cam.H)
        return gs::set_error(GS_EINVAL, "the image size is fixed at gs_raster_create");
    GS_TRY(check_camera(*c));
    set_camera(r, *c);
    r->have_forward = false;
    return GS_OK;
} GS_ABI_CATCH

extern "C" gs_status gs_raster_forward(gs_raster* r, const float* x, const float* colours, float* image, void* stream) try {
    gs::clear_error();
    if (!r || !x || !colours || !image) return gs::set_error(GS_EINVAL, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    GS_CUDA(cudaMemcpyAsync(r->x.p, x, 12 * (size_t)r->N, cudaMemcpyDeviceToDevice, s));
    GS_CUDA(cudaMemcpyAsync(r->col.p, colours, 12 * (size_t)r->N, cudaMemcpyDeviceToDevice, s));
    if (r->F > 0)
        k_rs_setup<<<(r->F + 127) / 128, 128, 0, s>>>((const float*)r->x.p, (const int*)r->faces.p, r->F, r->cam,
                                                      r->sp, (TriScr*)r->tri.p, (short4*)r->boxes.p);
    const dim3 sgrid(r->nsx * r->nsy, r->nch);
    int* counts = (int*)r->bin_counts.p;
    int* offsets = (int*)r->bin_offsets.p;
    int* flag = (int*)r->bin_flag.p;
    k_rs_bin_count<<<sgrid, 256, 0, s>>>((const short4*)r->boxes.p, r->F, r->chunk, r->nsx, r->cam.W, r->cam.H,
                                         counts);
    k_rs_bin_scan<<<1, 256, 0, s>>>(counts, r->nsx * r->nsy * kSub * r->nch, r->bin_cap, offsets, flag);
    k_rs_bin_fill<<<sgrid, 256, 0, s>>>((const short4*)r->boxes.p, r->F, r->chunk, r->nsx, r->cam.W, r->cam.H,
                                        offsets, flag, (int*)r->bin_lists.p);
    const dim3 grid((r->cam.W + kTile - 1) / kTile, (r->cam.H + kTile - 1) / kTile);
    k_rs_forward<<<grid, kTileThreads, 0, s>>>((const TriScr*)r->tri.p, (const short4*)r->boxes.p, r->F, counts,
                                               offsets, flag,
                                               (const int*)r->bin_lists.p, r->nsx, r->nch, (const float*)r->col.p,
                                               r->cam, r->sp, (float4*)image, (float4*)r->img.p, (float4*)r->aux.p);
    GS_CUDA(cudaGetLastError());
    r->have_forward = true;
    return GS_OK;
} GS_ABI_CATCH

extern "C" gs_status gs_raster_backward(gs_raster* r, const float* dL_dimage, float* dL_dx, float* dL_dcolours,
                                        void* stream) try {
    gs::clear_error();
    if (!r || !dL_dimage) return gs::set_error(GS_EINVAL, "null argument");
    if (!r->have_forward) return gs::set_error(GS_ESTATE, "gs_raster_backward needs a gs_raster_forward first");
    cudaStream_t s = (cudaStream_t)stream;
    if (r->F > 0) {
        constexpr int kWarps = 8;
        k_rs_backward<<<(r->F + kWarps - 1) / kWarps, 32 * kWarps, 0, s>>>(
            (const TriScr*)r->tri.p, r->F, (const float*)r->col.p, r->cam, r->sp, (const float4*)r->img.p,
            (const float4*)r->aux.p, (const float4*)dL_dimage, (TriGrad*)r->tgrad.p);
    }
    if (dL_dx || dL_dcolours)
        k_rs_vertex<<<(r->N + 127) / 128, 128, 0, s>>>((const int*)r->rowptr.p, (const int*)r->entries.p,
                                                       (const TriGrad*)r->tgrad.p, (const float*)r->x.p, r->cam,
                                                       r->N, dL_dx, dL_dcolours);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
} GS_ABI_CATCH
