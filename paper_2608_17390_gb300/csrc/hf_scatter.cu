// hf_scatter.cu -- the paper's Scattered method (its Section 3: the original
// engine's object-order painter recast as a parallel atomic scatter), as a
// comparison renderer for the exact cast.
//
// Per camera, a grid of nu x nv samples covers a camera-aligned ground
// footprint (longitudinal coordinate s along the camera's horizontal forward,
// quadratically warped so samples crowd near the camera; lateral coordinate u
// along its right vector, |u| <= u_min + k_lat |s|: a trapezoid).  Each sample walks the
// column of the cell under it -- nz points from the floor top down to 0, and
// for a slab nz points from its top down to its underside -- projects each
// point with the integer camera basis (d = F + aR + bU), and keeps, per pixel,
// the minimum of (24-bit quantised Euclidean depth << 8 | material | layer << 3)
// with a 32-bit atomicMin (the paper's packing).  A resolve pass then turns
// each pixel's word into a depth, the cell under the reconstructed point, the
// layer and a colour.  Sampling leaves gaps where the footprint is sparse: the
// trade-off the paper measures with its coherence metric.
//
// All arithmetic is float32, round to nearest, no fused multiply-add, in a
// fixed order, so the result is reproducible bit for bit (the packed screen
// does not depend on the order of the atomics: min is order-free).
#include <cuda_runtime.h>

#include "hf_internal.h"

namespace hf {
namespace {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr float kQMax = 16777215.0f;  // 2^24 - 1
constexpr int kScatterThreads = 256;

// float32 camera constants, computed in the definition's order
struct ScatterCam {
    float ox, oy, oz;
    float Fx, Fy, Fz, Rx, Ry, Rz, Ux, Uy, Uz;
    float cF, cR, cU;
    float rhx, rhy, fhx, fhy;
};

__device__ __forceinline__ float inv_sq(float x, float y, float z) {
    return __fdiv_rn(1.0f, __fadd_rn(__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)), __fmul_rn(z, z)));
}

__device__ __forceinline__ ScatterCam scatter_cam(const CamDev &c) {
    ScatterCam k;
    const float inv_s = 1.0f / 65536.0f;
    k.ox = __fmul_rn(__int2float_rn(c.o[0]), inv_s);
    k.oy = __fmul_rn(__int2float_rn(c.o[1]), inv_s);
    k.oz = __fmul_rn(__int2float_rn(c.o[2]), inv_s);
    k.Fx = (float)c.F[0];  // |components| < 2^21: exact
    k.Fy = (float)c.F[1];
    k.Fz = (float)c.F[2];
    k.Rx = (float)c.R[0];
    k.Ry = (float)c.R[1];
    k.Rz = (float)c.R[2];
    k.Ux = (float)c.U[0];
    k.Uy = (float)c.U[1];
    k.Uz = (float)c.U[2];
    k.cF = inv_sq(k.Fx, k.Fy, k.Fz);
    k.cR = inv_sq(k.Rx, k.Ry, k.Rz);
    k.cU = inv_sq(k.Ux, k.Uy, k.Uz);
    const float lr = __fsqrt_rn(__fadd_rn(__fmul_rn(k.Rx, k.Rx), __fmul_rn(k.Ry, k.Ry)));
    k.rhx = __fdiv_rn(k.Rx, lr);
    k.rhy = __fdiv_rn(k.Ry, lr);
    k.fhx = -k.rhy;
    k.fhy = k.rhx;
    return k;
}

__device__ __forceinline__ float dot3(float ax, float ay, float az, float bx, float by, float bz) {
    return __fadd_rn(__fadd_rn(__fmul_rn(ax, bx), __fmul_rn(ay, by)), __fmul_rn(az, bz));
}

// The parts of a point's view-space products that do not depend on its
// height: for v = (vx, vy, vz), dot3(v, a) = (vx ax + vy ay) + vz az, and the
// bracket is the same for every point of one column.
struct ColumnPartials {
    float vx, vy, pf, pr, pu, pd;
};

__device__ __forceinline__ ColumnPartials column_partials(const ScatterCam &k, float x, float y) {
    ColumnPartials c;
    c.vx = __fsub_rn(x, k.ox);
    c.vy = __fsub_rn(y, k.oy);
    c.pf = __fadd_rn(__fmul_rn(c.vx, k.Fx), __fmul_rn(c.vy, k.Fy));
    c.pr = __fadd_rn(__fmul_rn(c.vx, k.Rx), __fmul_rn(c.vy, k.Ry));
    c.pu = __fadd_rn(__fmul_rn(c.vx, k.Ux), __fmul_rn(c.vy, k.Uy));
    c.pd = __fadd_rn(__fmul_rn(c.vx, c.vx), __fmul_rn(c.vy, c.vy));
    return c;
}

// Packed depth word of a point without its type, or false when the point is
// behind the camera or outside the image.  The same operations, in the same
// order, as dot3 over the full vectors.
__device__ __forceinline__ bool project(const ScatterCam &k, const CamDev &c, float qscale,
                                        const ColumnPartials &cp, float z, uint32_t &pix,
                                        uint32_t &q) {
    const float vz = __fsub_rn(z, k.oz);
    const float vf = __fadd_rn(cp.pf, __fmul_rn(vz, k.Fz));
    if (!(vf > 0.0f)) return false;
    const float vr = __fadd_rn(cp.pr, __fmul_rn(vz, k.Rz));
    const float vu = __fadd_rn(cp.pu, __fmul_rn(vz, k.Uz));
    const float den = __fmul_rn(vf, k.cF);
    const float a = __fdiv_rn(__fmul_rn(vr, k.cR), den);
    const float b = __fdiv_rn(__fmul_rn(vu, k.cU), den);
    const float wf = (float)c.w, hf = (float)c.h;
    const float pxf = floorf(__fmul_rn(__fadd_rn(a, wf), 0.5f));
    const float pyf = floorf(__fmul_rn(__fsub_rn(hf, b), 0.5f));
    if (!(pxf >= 0.0f && pxf < wf && pyf >= 0.0f && pyf < hf)) return false;
    const float d = __fsqrt_rn(__fadd_rn(cp.pd, __fmul_rn(vz, vz)));
    q = __float2uint_rz(fminf(__fmul_rn(d, qscale), kQMax));
    pix = (uint32_t)pyf * c.w + (uint32_t)pxf;
    return true;
}

// column fractions m / (nz - 1) held in shared memory up to this count
constexpr int kScatterFracTable = 256;

__global__ void k_scatter_clear(const RenderParams p) {
    const CamDev &c = p.cams[blockIdx.y];
    const uint32_t n = c.w * c.h;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        c.hit_cell[i] = kEmpty;
}

__global__ void __launch_bounds__(kScatterThreads) k_scatter(const RenderParams p,
                                                             const ScatterParams s) {
    __shared__ float s_tm[kScatterFracTable];
    const float zden = (float)(s.nz - 1);
    for (uint32_t m = threadIdx.x; m < min(s.nz, (uint32_t)kScatterFracTable); m += blockDim.x)
        s_tm[m] = __fdiv_rn((float)m, zden);
    __syncthreads();
    const uint32_t cam = blockIdx.y;
    const CamDev &c = p.cams[cam];
    const float4 fp = reinterpret_cast<const float4 *>(p.cams + p.hdr->n_cams)[cam];
    const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= s.nu * s.nv) return;
    const uint32_t i = idx % s.nu, j = idx / s.nu;
    const ScatterCam k = scatter_cam(c);
    // footprint sample (i, j)
    const float t = __fdiv_rn(__fadd_rn((float)j, 0.5f), (float)s.nv);
    const float sl = __fadd_rn(fp.x, __fmul_rn(__fsub_rn(fp.y, fp.x), __fmul_rn(t, t)));
    const float half = __fadd_rn(fp.w, __fmul_rn(fabsf(sl), fp.z));
    const float ui = __fsub_rn(__fmul_rn(__fdiv_rn(__fadd_rn((float)i, 0.5f), (float)s.nu), 2.0f), 1.0f);
    const float u = __fmul_rn(half, ui);
    const float x = __fadd_rn(__fadd_rn(k.ox, __fmul_rn(sl, k.fhx)), __fmul_rn(u, k.rhx));
    const float y = __fadd_rn(__fadd_rn(k.oy, __fmul_rn(sl, k.fhy)), __fmul_rn(u, k.rhy));
    const float fx = floorf(x), fy = floorf(y);
    if (!(fx >= 0.0f && fx < (float)p.world.W && fy >= 0.0f && fy < (float)p.world.H)) return;
    const uint32_t node = level0_node(p.world, (int32_t)fx, (int32_t)fy);
    const uint32_t b0 = node & 0xFF, b1 = (node >> 8) & 0xFF, b2 = (node >> 16) & 0xFF;
    const uint32_t mat = (node >> 24) & 7;
    const bool slab = b2 > b0;  // node form: a slab exactly when its top is above the floor
    const float h0 = (float)b0, h1 = (float)b1, h2 = (float)b2;
    const float qscale = __fdiv_rn(kQMax, s.depth_max);
    const ColumnPartials cp = column_partials(k, x, y);
    uint32_t *buf = c.hit_cell;
    for (uint32_t m = 0; m < s.nz; ++m) {
        const float tm = m < (uint32_t)kScatterFracTable ? s_tm[m] : __fdiv_rn((float)m, zden);
        uint32_t pix, q;
        if (project(k, c, qscale, cp, __fsub_rn(h0, __fmul_rn(h0, tm)), pix, q))
            atomicMin(buf + pix, (q << 8) | mat);
        if (slab && project(k, c, qscale, cp, __fadd_rn(h2, __fmul_rn(__fsub_rn(h1, h2), tm)),
                            pix, q))
            atomicMin(buf + pix, (q << 8) | mat | 8u);
    }
}

__global__ void k_scatter_resolve(const RenderParams p, const ScatterParams s) {
    const CamDev &c = p.cams[blockIdx.y];
    const uint32_t n = c.w * c.h;
    const uint32_t pix = blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= n) return;
    const uint32_t word = c.hit_cell[pix];
    if (word == kEmpty) {
        if (c.layer) c.layer[pix] = 255;
        if (c.face) c.face[pix] = kFaceMiss;
        if (c.depth) c.depth[pix] = __int_as_float(0x7f800000);
        if (c.rgba) c.rgba[pix] = kSkyColour;
        return;
    }
    const float depth = __fmul_rn((float)(word >> 8), __fdiv_rn(s.depth_max, kQMax));
    const int32_t px = (int32_t)(pix % c.w), py = (int32_t)(pix / c.w);
    const int32_t a = 2 * px + 1 - (int32_t)c.w, b = (int32_t)c.h - 1 - 2 * py;
    const float dx = (float)(c.F[0] + a * c.R[0] + b * c.U[0]);
    const float dy = (float)(c.F[1] + a * c.R[1] + b * c.U[1]);
    const float dz = (float)(c.F[2] + a * c.R[2] + b * c.U[2]);
    const float dl = __fsqrt_rn(dot3(dx, dy, dz, dx, dy, dz));
    const float kk = __fdiv_rn(depth, dl);
    const float ox = __fmul_rn(__int2float_rn(c.o[0]), 1.0f / 65536.0f);
    const float oy = __fmul_rn(__int2float_rn(c.o[1]), 1.0f / 65536.0f);
    const float xw = __fadd_rn(ox, __fmul_rn(dx, kk)), yw = __fadd_rn(oy, __fmul_rn(dy, kk));
    const float cx = fminf(fmaxf(floorf(xw), 0.0f), (float)(p.world.W - 1));
    const float cy = fminf(fmaxf(floorf(yw), 0.0f), (float)(p.world.H - 1));
    c.hit_cell[pix] = (uint32_t)cy * (uint32_t)p.world.W + (uint32_t)cx;
    if (c.layer) c.layer[pix] = (uint8_t)((word >> 3) & 1);
    if (c.face) c.face[pix] = kFacePZ;
    if (c.depth) c.depth[pix] = depth;
    if (c.rgba) c.rgba[pix] = s.colour[word & 7];
}

}  // namespace

int launch_scatter(const RenderParams &p, const ScatterParams &s, uint32_t n_cams, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t px_blocks = (s.max_pixels + kScatterThreads - 1) / kScatterThreads;
    k_scatter_clear<<<dim3(px_blocks < 1024 ? px_blocks : 1024, n_cams), kScatterThreads, 0, st>>>(p);
    const uint32_t samples = s.nu * s.nv;
    k_scatter<<<dim3((samples + kScatterThreads - 1) / kScatterThreads, n_cams), kScatterThreads, 0,
                st>>>(p, s);
    if (!s.raw)
        k_scatter_resolve<<<dim3(px_blocks, n_cams), kScatterThreads, 0, st>>>(p, s);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace hf
