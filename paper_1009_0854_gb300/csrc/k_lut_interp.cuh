// k_lut_interp.cuh -- the interpolation kernels of the four LUT methods
// (Section "Comparison with 3D Lookup Table Interpolation Methods") and
// their launchers, for one method per object: included only by
// k_lut_inst.cu, which the build compiles once per method.  Extraction,
// node placement and the evaluation forms are described in k_lut.cu.
#pragma once

#include <atomic>

#include "engine.cuh"
#include "internal.h"

namespace mact {

// ---------------------------------------------------------- interpolation

// Extraction along one axis for code v (node placement as in Kang's LUT
// methods, which the paper follows): s = v (n-1), idx = s div 255,
// rem = s mod 255, and v = 255 uses idx = n-2, rem = 255 -- i.e. idx is
// clamped to n-2 and rem = s - 255 idx; the fraction is rem * fl(1/255).
// Computed in registers: a per-code table in shared memory measured slower
// (lanes four codes apart, as in the cube's B channel, hit the same banks).
struct LocEntry {
    int idx;
    float f;
};

__device__ __forceinline__ LocEntry loc_entry(uint32_t v, int n)
{
    const int s = (int)v * (n - 1);
    const int idx = min(s / 255, n - 2);
    const int rem = s - 255 * idx;
    // rem * fl(1/255): strictly increasing in rem, so comparing fractions
    // orders cells exactly as the integer remainders do
    return LocEntry{idx, (float)rem * (1.0f / 255.0f)};
}

// A node value (three channels) as one FP32 pair and a scalar.  With PK each
// elementwise step is one packed f32x2 instruction plus one scalar
// instruction, rounded exactly like three scalar ones; without it, three
// scalar instructions.  Measured on the 2^24 cube, packing pays for the
// tetrahedral method (309 vs 297 Gpix/s at 17^3) and the 33^3 pyramid
// (245 vs 238); for trilinear and prism it was 2-6% slower and it made the
// 17^3 pyramid spill (pair registers must be aligned, which raises register
// pressure).
struct V3 {
    float2 xy;
    float z;
};
template <bool PK>
__device__ __forceinline__ V3 v3sub(V3 a, V3 b)
{
    if (PK) return V3{sub2(a.xy, b.xy), a.z - b.z};
    return V3{make_float2(a.xy.x - b.xy.x, a.xy.y - b.xy.y), a.z - b.z};
}
template <bool PK>
__device__ __forceinline__ V3 v3add(V3 a, V3 b)
{
    if (PK) return V3{add2(a.xy, b.xy), a.z + b.z};
    return V3{make_float2(a.xy.x + b.xy.x, a.xy.y + b.xy.y), a.z + b.z};
}
// d * w + c, each channel one fused multiply-add
template <bool PK>
__device__ __forceinline__ V3 v3fma(V3 d, float w, V3 c)
{
    if (PK) return V3{fma2(d.xy, make_float2(w, w), c.xy), fmaf(d.z, w, c.z)};
    return V3{make_float2(fmaf(d.xy.x, w, c.xy.x), fmaf(d.xy.y, w, c.xy.y)), fmaf(d.z, w, c.z)};
}
// a + w (b - a), rounded as fmaf(b - a, w, a)
template <bool PK>
__device__ __forceinline__ V3 v3lerp(V3 a, V3 b, float w) { return v3fma<PK>(v3sub<PK>(b, a), w, a); }

// Where a kernel reads its nodes: float4 nodes in shared memory, float4
// nodes (or caching-layout records) in global memory, or the caller's packed
// float3 nodes in global memory.
enum { kSrcShared4 = 0, kSrcGlobal4 = 1, kSrcGlobal3 = 2 };

// Node i of the array at lut.  With NARROW a float4 node's padding float is
// not read (an 8-byte and a 4-byte load instead of one 16-byte load): fewer
// live registers for the same values; measured on GB300 it pays only for the
// pyramid (5 nodes, the most register-hungry selection).
template <int SRC, bool NARROW = false>
__device__ __forceinline__ V3 fetch(const float *lut, int i)
{
    if constexpr (SRC == kSrcGlobal3) {
        const float *p = lut + 3 * i;
        return V3{make_float2(__ldg(p), __ldg(p + 1)), __ldg(p + 2)};
    } else if constexpr (!NARROW) {
        const float4 *p = reinterpret_cast<const float4 *>(lut) + i;
        const float4 v = SRC == kSrcShared4 ? *p : __ldg(p);
        return V3{make_float2(v.x, v.y), v.z};
    } else {
        const float *f = lut + 4 * i;
        if constexpr (SRC == kSrcShared4)
            return V3{*reinterpret_cast<const float2 *>(f), f[2]};
        else
            return V3{__ldg(reinterpret_cast<const float2 *>(f)), __ldg(f + 2)};
    }
}

// Node-array geometry: the strides of R and G (B is 1) and an origin
// subtracted from every node index.  Compile-time (the whole n^3 array, n = N)
// unless RT: then per launch or per tile (a staged sub-box of the lattice).
template <int N, bool RT>
struct Geo {
    int sr, sg, org;
    __device__ __forceinline__ int r() const { return RT ? sr : N * N; }
    __device__ __forceinline__ int g() const { return RT ? sg : N; }
    __device__ __forceinline__ int o() const { return RT ? org : 0; }
};

// Nodes each method reads from its cell.
template <int METHOD>
struct NodeCount {
    static constexpr int K = METHOD == MACT_TRILINEAR ? 8 : METHOD == MACT_PRISM ? 6 : METHOD == MACT_PYRAMID ? 5 : 4;
};

// Extraction result of one pixel: the lower-corner node index in the whole
// lattice (for the selection id), the index into the node array read, the
// simplex, the node offsets (relative to the lower corner) and the three
// weights the interpolation formula uses.
template <int METHOD>
struct Sel {
    int base;
    int addr;
    int simplex;
    int off[NodeCount<METHOD>::K];
    float w0, w1, w2;
};

// CACHED: nodes come from the per-cell records of the caching layout (addr is
// the cell's first slot; node offsets become record slots and the value is
// c000 + the interpolation of the differences).
template <int METHOD, int SRC, int N, bool RT, bool CACHED = false>
struct OpLut {
    static constexpr int K = NodeCount<METHOD>::K;
    // packed pairs (see V3): tetrahedral, and the pyramid read from global
    // memory (+3% at 33^3; in shared memory its pairs spilled)
    static constexpr bool PK = (METHOD == MACT_TETRA || (METHOD == MACT_PYRAMID && SRC == kSrcGlobal4)) && !CACHED;
    const float *lut;          // node array (float4 nodes or records, or float3 nodes)
    int n;                     // lattice size (runtime when N == 0)
    Geo<N, RT> geo;

    __device__ __forceinline__ int nn() const { return N > 0 ? N : n; }

    __device__ __forceinline__ Sel<METHOD> select(uint32_t r, uint32_t g, uint32_t b) const
    {
        const int n_ = nn();
        const LocEntry er = loc_entry(r, n_), eg = loc_entry(g, n_), eb = loc_entry(b, n_);
        const float fr = er.f, fg = eg.f, fb = eb.f;
        Sel<METHOD> q;
        q.base = (er.idx * n_ + eg.idx) * n_ + eb.idx;
        // node strides, or record slot strides in the caching layout
        int sR, sG;
        if (CACHED) {
            sR = 4;
            sG = 2;
            q.addr = ((er.idx * (n_ - 1) + eg.idx) * (n_ - 1) + eb.idx) * 8;
        } else {
            sR = geo.r();
            sG = geo.g();
            q.addr = er.idx * sR + eg.idx * sG + eb.idx - geo.o();
        }
        const int sB = 1;
        if (METHOD == MACT_TRILINEAR) {
            const int o[8] = {0, sB, sG, sG + sB, sR, sR + sB, sR + sG, sR + sG + sB};
#pragma unroll
            for (int k = 0; k < 8; ++k) q.off[k] = o[k];
            q.simplex = 0;
            q.w0 = fb; q.w1 = fg; q.w2 = fr;
        } else if (METHOD == MACT_PRISM) {
            // prism axis R; triangle in the G-B face chosen by rem_G >= rem_B
            const bool lo = fg >= fb;
            const int oe = lo ? sG : sB;   // c010 or c001
            const int o[6] = {0, sR, sG + sB, sR + sG + sB, oe, sR + oe};
#pragma unroll
            for (int k = 0; k < 6; ++k) q.off[k] = o[k];
            q.simplex = lo ? 0 : 1;
            q.w0 = lo ? fg : fb; q.w1 = lo ? fb : fg; q.w2 = fr;
        } else if (METHOD == MACT_PYRAMID) {
            // apex c111; base on the face of the smallest fraction (B, then G, then R)
            int oX, oY;
            if (fb <= fr && fb <= fg) { oX = sR; oY = sG; q.w0 = fr; q.w1 = fg; q.w2 = fb; q.simplex = 0; }
            else if (fg <= fr && fg <= fb) { oX = sR; oY = sB; q.w0 = fr; q.w1 = fb; q.w2 = fg; q.simplex = 1; }
            else { oX = sG; oY = sB; q.w0 = fg; q.w1 = fb; q.w2 = fr; q.simplex = 2; }
            const int o[5] = {0, sR + sG + sB, oX, oY, oX + oY};
#pragma unroll
            for (int k = 0; k < 5; ++k) q.off[k] = o[k];
        } else {
            // tetrahedral: path from c000 along the axes in decreasing fraction
            int o1, o2;
            if (fr >= fg && fg >= fb)      { o1 = sR; o2 = sR + sG; q.w0 = fr; q.w1 = fg; q.w2 = fb; q.simplex = 0; }
            else if (fr >= fb && fb > fg)  { o1 = sR; o2 = sR + sB; q.w0 = fr; q.w1 = fb; q.w2 = fg; q.simplex = 1; }
            else if (fb > fr && fr >= fg)  { o1 = sB; o2 = sR + sB; q.w0 = fb; q.w1 = fr; q.w2 = fg; q.simplex = 2; }
            else if (fg > fr && fr >= fb)  { o1 = sG; o2 = sR + sG; q.w0 = fg; q.w1 = fr; q.w2 = fb; q.simplex = 3; }
            else if (fg >= fb && fb > fr)  { o1 = sG; o2 = sG + sB; q.w0 = fg; q.w1 = fb; q.w2 = fr; q.simplex = 4; }
            else                           { o1 = sB; o2 = sG + sB; q.w0 = fb; q.w1 = fg; q.w2 = fr; q.simplex = 5; }
            const int o[4] = {0, o1, o2, sR + sG + sB};
#pragma unroll
            for (int k = 0; k < 4; ++k) q.off[k] = o[k];
        }
        return q;
    }

    __device__ __forceinline__ void load(const Sel<METHOD> &q, V3 (&nd)[K]) const
    {
#pragma unroll
        for (int k = 0; k < K; ++k) nd[k] = fetch<SRC, METHOD == MACT_PYRAMID && SRC != kSrcGlobal3>(lut, q.addr + q.off[k]);
    }

    // value from the loaded nodes: directly, or c000 + interpolated differences
    __device__ __forceinline__ static V3 value(const V3 (&nd)[K], const Sel<METHOD> &q)
    {
        if (!CACHED) return interp(nd, q);
        V3 d[K];
        d[0] = V3{make_float2(0.f, 0.f), 0.f};
#pragma unroll
        for (int k = 1; k < K; ++k) d[k] = nd[k];
        return v3add<PK>(nd[0], interp(d, q));
    }

    __device__ __forceinline__ static V3 interp(const V3 (&nd)[K], const Sel<METHOD> &q)
    {
        if (METHOD == MACT_TRILINEAR) {
            // repeated linear interpolation along B, then G, then R
            // nd: c000 c001 c010 c011 c100 c101 c110 c111
            const V3 c00 = v3lerp<PK>(nd[0], nd[1], q.w0);
            const V3 c01 = v3lerp<PK>(nd[2], nd[3], q.w0);
            const V3 c10 = v3lerp<PK>(nd[4], nd[5], q.w0);
            const V3 c11 = v3lerp<PK>(nd[6], nd[7], q.w0);
            const V3 c0 = v3lerp<PK>(c00, c01, q.w1);
            const V3 c1 = v3lerp<PK>(c10, c11, q.w1);
            return v3lerp<PK>(c0, c1, q.w2);
        } else if (METHOD == MACT_PRISM) {
            // nd: c000 c100 c011 c111 ce0 ce1; triangle at R = 0 and R = 1, then linear in R
            const V3 t0 = v3fma<PK>(v3sub<PK>(nd[2], nd[4]), q.w1, v3lerp<PK>(nd[0], nd[4], q.w0));
            const V3 t1 = v3fma<PK>(v3sub<PK>(nd[3], nd[5]), q.w1, v3lerp<PK>(nd[1], nd[5], q.w0));
            return v3lerp<PK>(t0, t1, q.w2);
        } else if (METHOD == MACT_PYRAMID) {
            // nd: c000 c111 cX cY cA;
            // c000 + (c111-cA) fZ + (cX-c000) fX + (cY-c000) fY + (cA-cX-cY+c000) fX fY
            const V3 cross = v3add<PK>(v3sub<PK>(v3sub<PK>(nd[4], nd[2]), nd[3]), nd[0]);
            V3 acc = v3fma<PK>(v3sub<PK>(nd[1], nd[4]), q.w2, nd[0]);
            acc = v3fma<PK>(v3sub<PK>(nd[2], nd[0]), q.w0, acc);
            acc = v3fma<PK>(v3sub<PK>(nd[3], nd[0]), q.w1, acc);
            return v3fma<PK>(cross, q.w0 * q.w1, acc);
        } else {
            // nd: c000 c1 c2 c111
            V3 acc = v3lerp<PK>(nd[0], nd[1], q.w0);
            acc = v3fma<PK>(v3sub<PK>(nd[2], nd[1]), q.w1, acc);
            return v3fma<PK>(v3sub<PK>(nd[3], nd[2]), q.w2, acc);
        }
    }

    __device__ __forceinline__ int operator()(uint32_t r, uint32_t g, uint32_t b, float &o0, float &o1,
                                              float &o2) const
    {
        const Sel<METHOD> q = select(r, g, b);
        V3 nd[K];
        load(q, nd);
        const V3 v = value(nd, q);
        o0 = v.xy.x;
        o1 = v.xy.y;
        o2 = v.z;
        return q.base * 8 + q.simplex;
    }
};

// ------------------------------------------------ whole LUT in shared memory
// n <= 17: every CTA stages the LUT as float4 nodes (17^3 x 16 B = 78.6 KB;
// from the caller's packed float3 nodes, or from a float4 copy), so a node is
// one 16-byte shared load at an immediate offset from the cell's lower
// corner.
template <int THREADS, int MINB, int METHOD, int N, bool SEL>
__global__ void __launch_bounds__(THREADS, MINB)
k_lut_whole(const __grid_constant__ ImageDesc im, const float *__restrict__ lut, const float4 *__restrict__ lut4,
            int n, int32_t *sel, int64_t ntiles)
{
    extern __shared__ float4 slut[];
    __shared__ uint4 sbuf[TileShape<THREADS>::vecs];
    const int nodes = n * n * n;
    if (lut4) {
        for (int i = threadIdx.x; i < nodes; i += THREADS) slut[i] = lut4[i];
    } else {
        for (int i = threadIdx.x; i < nodes; i += THREADS)
            slut[i] = make_float4(lut[3 * i], lut[3 * i + 1], lut[3 * i + 2], 0.0f);
    }
    OpLut<METHOD, kSrcShared4, N, N == 0> op;
    op.lut = reinterpret_cast<const float *>(slut);
    op.n = n;
    op.geo = {n * n, n, 0};
    run_image<THREADS, float, SEL>(im, ntiles, op, sbuf, sel);   // its first barrier orders the staging
}

// ------------------------------------------ float4 nodes in global memory
// Nodes read through L1 from a float4 copy of the LUT (one 16-byte load per
// node), for LUTs too large for shared memory.
template <int THREADS, int MINB, int METHOD, int N, bool SEL>
__global__ void __launch_bounds__(THREADS, MINB)
k_lut_global(const __grid_constant__ ImageDesc im, const float4 *__restrict__ lut4, int n, int32_t *sel,
             int64_t ntiles)
{
    __shared__ uint4 sbuf[TileShape<THREADS>::vecs];
    OpLut<METHOD, kSrcGlobal4, N, N == 0> op;
    op.lut = reinterpret_cast<const float *>(lut4);
    op.n = n;
    op.geo = {n * n, n, 0};
    run_image<THREADS, float, SEL>(im, ntiles, op, sbuf, sel);
}

// ------------------------------------- trilinear from B-edge records
// For LUTs read from global memory, trilinear interpolation fetches its 8
// nodes as the 4 edges along B of its cell (xy record: the two nodes' x and y,
// 16 bytes; z record: their z, 8 bytes): 4 + 4 loads of 96 bytes instead of 8
// loads of 128, which measured 25% faster on the 2^24-colour cube for a 33^3
// LUT (the kernel is bound by the L1 data path).  Repeated linear
// interpolation along B, then G, then R, each lerp rounded as
// fmaf(b - a, w, a); x and y run as packed FP32 pairs.
template <int N>
struct OpEdge {
    const float4 *xy;
    const float2 *z;
    int n;
    __device__ __forceinline__ int operator()(uint32_t r, uint32_t g, uint32_t b, float &o0, float &o1,
                                              float &o2) const
    {
        const int n_ = N > 0 ? N : n;
        const LocEntry er = loc_entry(r, n_), eg = loc_entry(g, n_), eb = loc_entry(b, n_);
        const int base = (er.idx * n_ + eg.idx) * n_ + eb.idx;
        const int sG = n_, sR = n_ * n_;
        // edges at (R, G) offsets (0, 0), (0, 1), (1, 0), (1, 1)
        const float4 a0 = __ldg(xy + base), a1 = __ldg(xy + base + sG), a2 = __ldg(xy + base + sR),
                     a3 = __ldg(xy + base + sR + sG);
        const float2 z0 = __ldg(z + base), z1 = __ldg(z + base + sG), z2 = __ldg(z + base + sR),
                     z3 = __ldg(z + base + sR + sG);
        const float2 wb = make_float2(eb.f, eb.f);
        const float2 c00 = fma2(sub2(make_float2(a0.z, a0.w), make_float2(a0.x, a0.y)), wb, make_float2(a0.x, a0.y));
        const float2 c01 = fma2(sub2(make_float2(a1.z, a1.w), make_float2(a1.x, a1.y)), wb, make_float2(a1.x, a1.y));
        const float2 c10 = fma2(sub2(make_float2(a2.z, a2.w), make_float2(a2.x, a2.y)), wb, make_float2(a2.x, a2.y));
        const float2 c11 = fma2(sub2(make_float2(a3.z, a3.w), make_float2(a3.x, a3.y)), wb, make_float2(a3.x, a3.y));
        const float d00 = fmaf(z0.y - z0.x, eb.f, z0.x), d01 = fmaf(z1.y - z1.x, eb.f, z1.x);
        const float d10 = fmaf(z2.y - z2.x, eb.f, z2.x), d11 = fmaf(z3.y - z3.x, eb.f, z3.x);
        const float2 wg = make_float2(eg.f, eg.f);
        const float2 c0 = fma2(sub2(c01, c00), wg, c00), c1 = fma2(sub2(c11, c10), wg, c10);
        const float d0 = fmaf(d01 - d00, eg.f, d00), d1 = fmaf(d11 - d10, eg.f, d10);
        const float2 v = fma2(sub2(c1, c0), make_float2(er.f, er.f), c0);
        o0 = v.x;
        o1 = v.y;
        o2 = fmaf(d1 - d0, er.f, d0);
        return base * 8;   // trilinear: one simplex
    }
};

// Both ends of the edge record at i: a = node i, b = the next node along the
// record's axis.
__device__ __forceinline__ void edge(const float4 *xy, const float2 *z, int i, V3 &a, V3 &b)
{
    const float4 p = __ldg(xy + i);
    const float2 q = __ldg(z + i);
    a = V3{make_float2(p.x, p.y), q.x};
    b = V3{make_float2(p.z, p.w), q.y};
}

// Prism and pyramid from the packed layout: the same selection and the same
// interpolation arithmetic as OpLut (so the same bits); only the node loads
// differ.  Prism reads its 6 nodes as 3 edges along R (c000-c100, c011-c111,
// ce0-ce1): 72 bytes in 6 loads instead of 96 (+19% on the cube at 33^3).
// The pyramid reads single nodes from the dense xy and z planes: 12 bytes in
// two loads per node, where neighbouring pixels' nodes share 25% fewer
// sectors than in the 16-byte node array (+4%).  Measured and not kept:
// the pyramid's five nodes as two edges and a node (14% slower: the per-pixel
// case selects cost more than the bytes saved), and the tetrahedral method
// from the planes (7% slower on the cube, 45% on noise).
template <int METHOD, int N>
struct OpLutPacked {
    using Base = OpLut<METHOD, kSrcGlobal4, N, N == 0>;
    static constexpr int K = NodeCount<METHOD>::K;
    Base base;
    PackedLut pk;

    __device__ __forceinline__ int operator()(uint32_t r, uint32_t g, uint32_t b, float &o0, float &o1,
                                              float &o2) const
    {
        const Sel<METHOD> q = base.select(r, g, b);
        V3 nd[K];
        if constexpr (METHOD == MACT_PRISM) {
            // off: 0, sR, sG + sB, sR + sG + sB, oe, sR + oe
            edge(pk.rxy, pk.rz, q.addr + q.off[0], nd[0], nd[1]);
            edge(pk.rxy, pk.rz, q.addr + q.off[2], nd[2], nd[3]);
            edge(pk.rxy, pk.rz, q.addr + q.off[4], nd[4], nd[5]);
        } else {
            // pyramid: single nodes from the dense planes, 8 + 4 bytes each
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int i = q.addr + q.off[k];
                nd[k] = V3{__ldg(pk.pxy + i), __ldg(pk.pz + i)};
            }
        }
        const V3 v = Base::value(nd, q);
        o0 = v.xy.x;
        o1 = v.xy.y;
        o2 = v.z;
        return q.base * 8 + q.simplex;
    }
};

template <int THREADS, int MINB, int METHOD, int N, bool SEL>
__global__ void __launch_bounds__(THREADS, MINB)
k_lut_packed(const __grid_constant__ ImageDesc im, const __grid_constant__ PackedLut pk, int n, int32_t *sel,
             int64_t ntiles)
{
    __shared__ uint4 sbuf[TileShape<THREADS>::vecs];
    OpLutPacked<METHOD, N> op;
    op.base.lut = reinterpret_cast<const float *>(pk.nodes);
    op.base.n = n;
    op.base.geo = {n * n, n, 0};
    op.pk = pk;
    run_image<THREADS, float, SEL>(im, ntiles, op, sbuf, sel);
}

template <int THREADS, int MINB, int N, bool SEL>
__global__ void __launch_bounds__(THREADS, MINB)
k_lut_edge(const __grid_constant__ ImageDesc im, const float4 *__restrict__ xy, const float2 *__restrict__ z, int n,
           int32_t *sel, int64_t ntiles)
{
    __shared__ uint4 sbuf[TileShape<THREADS>::vecs];
    const OpEdge<N> op{xy, z, n};
    run_image<THREADS, float, SEL>(im, ntiles, op, sbuf, sel);
}

// ------------------------------------------------------ caching layout
template <int THREADS, int MINB, int METHOD, int N, bool SEL>
__global__ void __launch_bounds__(THREADS, MINB)
k_lut_cached(const __grid_constant__ ImageDesc im, const float4 *__restrict__ cache, int n, int32_t *sel,
             int64_t ntiles)
{
    __shared__ uint4 sbuf[TileShape<THREADS>::vecs];
    OpLut<METHOD, kSrcGlobal4, N, N == 0, true> op;
    op.lut = reinterpret_cast<const float *>(cache);
    op.n = n;
    op.geo = {n * n, n, 0};
    run_image<THREADS, float, SEL>(im, ntiles, op, sbuf, sel);
}

// ------------------------------------------------------------- launchers

// Threads per CTA of the whole-LUT kernels (two CTAs per SM, each with its
// own staged copy of the LUT).  The register cap this leaves (128 at 256
// threads, 85 at 384) keeps the interpolators from spilling; measured on the
// 2^24 cube, 256 threads suit trilinear, prism and pyramid and 384 the
// tetrahedral method (512 threads, 64 registers, spilled: 11-21% slower).
template <int METHOD>
struct WholeThreads {
    static constexpr int value = METHOD == MACT_TETRA ? 384 : 256;
};


// Launch shape of the global-memory kernels: trilinear 256 threads x 3 CTAs
// (24 warps per SM, 80 registers); prism 128 x 6 (the same warps, 2-6% faster
// than 256 x 3 for it); pyramid and tetrahedral 128 x 7 (28 warps at 72
// registers: +4% over 128 x 6 on the 2^24 cube at 33^3, where the prism lost
// 2% and spilled).  A 64-register cap (32 warps) spilled and was 2-6% slower.
template <int METHOD>
struct GlobalShape {
    static constexpr int threads = METHOD == MACT_TRILINEAR ? 256 : 128;
    static constexpr int ctas = METHOD == MACT_TRILINEAR ? 3 : METHOD == MACT_PRISM ? 6 : 7;
};

template <class Kern>
static int occupancy(Kern kern, int threads, size_t smem)
{
    int o = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, threads, smem);
    return (e != cudaSuccess || o <= 0) ? 1 : o;
}

// Sets a kernel's dynamic shared memory limit once per device (a bit per
// device ordinal < 64; concurrent first launches set the same value).
template <class Kern>
static cudaError_t smem_attr(std::atomic<uint64_t> &done, int device, Kern kern, int bytes)
{
    const uint64_t bit = 1ull << (device & 63);
    if ((done.load(std::memory_order_acquire) & bit) != 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

static ImageDesc row_desc(const uint8_t *rgb, float *const out[3], int64_t npix, int tile_px)
{
    ImageDesc im{};
    im.rgb = rgb;
    for (int c = 0; c < 3; ++c) im.out[c] = out[c];
    im.width = npix;
    im.height = 1;
    im.pitch = 3 * npix;
    im.opitch = npix;
    im.space = MACT_CIELAB;
    im.dtype = MACT_F32;
    im.tiles_per_row = (npix + tile_px - 1) / tile_px;
    return im;
}

template <int METHOD, int N, bool SEL>
static cudaError_t launch_whole(const mact_ctx &h, const float *lut, const float4 *lut4, int n, const uint8_t *rgb,
                                int64_t npix, float *const out[3], int32_t *sel, cudaStream_t s)
{
    constexpr int T = WholeThreads<METHOD>::value;
    const ImageDesc im = row_desc(rgb, out, npix, TileShape<T>::px);
    const int64_t nt = im.tiles_per_row;
    auto kern = k_lut_whole<T, 2, METHOD, N, SEL>;
    const size_t smem = (size_t)n * n * n * sizeof(float4);
    static std::atomic<uint64_t> attr{0};
    static std::atomic<int> occ_cache[kLutSmemMaxN + 1];
    cudaError_t e = smem_attr(attr, h.device, kern, kLutSmemMaxN * kLutSmemMaxN * kLutSmemMaxN * (int)sizeof(float4));
    if (e != cudaSuccess) return e;
    int occ = occ_cache[n].load(std::memory_order_relaxed);
    if (occ == 0) {
        occ = occupancy(kern, T, smem);
        occ_cache[n].store(occ, std::memory_order_relaxed);
    }
    const int64_t cap = (int64_t)h.num_sms * occ;
    kern<<<(unsigned)(nt < cap ? nt : cap), T, smem, s>>>(im, lut, lut4, n, sel, nt);
    return cudaGetLastError();
}

template <int METHOD, int N, bool SEL>
static cudaError_t launch_global(const mact_ctx &h, const float4 *lut4, int n, const uint8_t *rgb, int64_t npix,
                                 float *const out[3], int32_t *sel, cudaStream_t s)
{
    constexpr int T = GlobalShape<METHOD>::threads;
    const ImageDesc im = row_desc(rgb, out, npix, TileShape<T>::px);
    const int64_t nt = im.tiles_per_row;
    auto kern = k_lut_global<T, GlobalShape<METHOD>::ctas, METHOD, N, SEL>;
    static std::atomic<int> occ_cache{0};
    int occ = occ_cache.load(std::memory_order_relaxed);
    if (occ == 0) {
        occ = occupancy(kern, T, 0);
        occ_cache.store(occ, std::memory_order_relaxed);
    }
    const int64_t cap = (int64_t)h.num_sms * occ;
    kern<<<(unsigned)(nt < cap ? nt : cap), T, 0, s>>>(im, lut4, n, sel, nt);
    return cudaGetLastError();
}

template <int METHOD, int N, bool SEL>
static cudaError_t launch_cached(const mact_ctx &h, const float4 *cache, int n, const uint8_t *rgb, int64_t npix,
                                 float *const out[3], int32_t *sel, cudaStream_t s)
{
    const ImageDesc im = row_desc(rgb, out, npix, TileShape<kThreads>::px);
    const int64_t nt = im.tiles_per_row;
    auto kern = k_lut_cached<kThreads, 4, METHOD, N, SEL>;
    static std::atomic<int> occ_cache{0};
    int occ = occ_cache.load(std::memory_order_relaxed);
    if (occ == 0) {
        occ = occupancy(kern, kThreads, 0);
        occ_cache.store(occ, std::memory_order_relaxed);
    }
    const int64_t cap = (int64_t)h.num_sms * occ;
    kern<<<(unsigned)(nt < cap ? nt : cap), kThreads, 0, s>>>(im, cache, n, sel, nt);
    return cudaGetLastError();
}

// packed: the layout of launch_lut_pack (nodes, then the B-edge records)
template <int N, bool SEL>
static cudaError_t launch_edge(const mact_ctx &h, const float4 *packed, int n, const uint8_t *rgb, int64_t npix,
                               float *const out[3], int32_t *sel, cudaStream_t s)
{
    constexpr int T = GlobalShape<MACT_TRILINEAR>::threads;
    const ImageDesc im = row_desc(rgb, out, npix, TileShape<T>::px);
    const int64_t nt = im.tiles_per_row;
    auto kern = k_lut_edge<T, GlobalShape<MACT_TRILINEAR>::ctas, N, SEL>;
    static std::atomic<int> occ_cache{0};
    int occ = occ_cache.load(std::memory_order_relaxed);
    if (occ == 0) {
        occ = occupancy(kern, T, 0);
        occ_cache.store(occ, std::memory_order_relaxed);
    }
    const int64_t cap = (int64_t)h.num_sms * occ;
    const PackedLut pk = packed_lut(packed, n);
    kern<<<(unsigned)(nt < cap ? nt : cap), T, 0, s>>>(im, pk.bxy, pk.bz, n, sel, nt);
    return cudaGetLastError();
}

template <int METHOD, int N, bool SEL>
static cudaError_t launch_packed(const mact_ctx &h, const float4 *packed, int n, const uint8_t *rgb, int64_t npix,
                                 float *const out[3], int32_t *sel, cudaStream_t s)
{
    constexpr int T = GlobalShape<METHOD>::threads;
    const ImageDesc im = row_desc(rgb, out, npix, TileShape<T>::px);
    const int64_t nt = im.tiles_per_row;
    auto kern = k_lut_packed<T, GlobalShape<METHOD>::ctas, METHOD, N, SEL>;
    static std::atomic<int> occ_cache{0};
    int occ = occ_cache.load(std::memory_order_relaxed);
    if (occ == 0) {
        occ = occupancy(kern, T, 0);
        occ_cache.store(occ, std::memory_order_relaxed);
    }
    const int64_t cap = (int64_t)h.num_sms * occ;
    kern<<<(unsigned)(nt < cap ? nt : cap), T, 0, s>>>(im, packed_lut(packed, n), n, sel, nt);
    return cudaGetLastError();
}

template <int METHOD, bool SEL>
cudaError_t lut_interp_method(const mact_ctx &h, const float *lut, const float4 *lut4, int n,
                                 const uint8_t *rgb, int64_t npix, float *const out[3], int32_t *sel, cudaStream_t s)
{
    if (n == 9) return launch_whole<METHOD, 9, SEL>(h, lut, lut4, n, rgb, npix, out, sel, s);
    if (n == 17) return launch_whole<METHOD, 17, SEL>(h, lut, lut4, n, rgb, npix, out, sel, s);
    if (n <= kLutSmemMaxN) return launch_whole<METHOD, 0, SEL>(h, lut, lut4, n, rgb, npix, out, sel, s);
    if constexpr (METHOD == MACT_TRILINEAR) {
        if (n == 33) return launch_edge<33, SEL>(h, lut4, n, rgb, npix, out, sel, s);
        return launch_edge<0, SEL>(h, lut4, n, rgb, npix, out, sel, s);
    } else if constexpr (METHOD == MACT_PRISM || METHOD == MACT_PYRAMID) {
        if (n == 33) return launch_packed<METHOD, 33, SEL>(h, lut4, n, rgb, npix, out, sel, s);
        return launch_packed<METHOD, 0, SEL>(h, lut4, n, rgb, npix, out, sel, s);
    } else {
        if (n == 33) return launch_global<METHOD, 33, SEL>(h, lut4, n, rgb, npix, out, sel, s);
        return launch_global<METHOD, 0, SEL>(h, lut4, n, rgb, npix, out, sel, s);
    }
}

template <int METHOD, bool SEL>
cudaError_t lut_cached_method(const mact_ctx &h, const float4 *cache, int n, const uint8_t *rgb, int64_t npix,
                                 float *const out[3], int32_t *sel, cudaStream_t s)
{
    if (n == 17) return launch_cached<METHOD, 17, SEL>(h, cache, n, rgb, npix, out, sel, s);
    if (n == 33) return launch_cached<METHOD, 33, SEL>(h, cache, n, rgb, npix, out, sel, s);
    return launch_cached<METHOD, 0, SEL>(h, cache, n, rgb, npix, out, sel, s);
}

}  // namespace mact

// Explicit instantiation of one method's entry points (inside namespace mact).
#define MACT_LUT_METHOD(METHOD)                                                                               \
    template cudaError_t lut_interp_method<METHOD, false>(const mact_ctx &, const float *, const float4 *, int, \
                                                          const uint8_t *, int64_t, float *const[3], int32_t *,   \
                                                          cudaStream_t);                                          \
    template cudaError_t lut_interp_method<METHOD, true>(const mact_ctx &, const float *, const float4 *, int,  \
                                                         const uint8_t *, int64_t, float *const[3], int32_t *,    \
                                                         cudaStream_t);                                           \
    template cudaError_t lut_cached_method<METHOD, false>(const mact_ctx &, const float4 *, int, const uint8_t *, \
                                                          int64_t, float *const[3], int32_t *, cudaStream_t);     \
    template cudaError_t lut_cached_method<METHOD, true>(const mact_ctx &, const float4 *, int, const uint8_t *,  \
                                                         int64_t, float *const[3], int32_t *, cudaStream_t);
