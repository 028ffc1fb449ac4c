// Mapping side of the path (Sec. III-B, Sec. IV-B-2 Remark 2): the exact
// Euclidean distance transform of an occupancy grid on the GPU, the
// robot-masked occupancy reset, and the update of a context's distance
// field from an occupancy grid.
//
// EDT: the separable three-pass squared transform along y, then x, then z,
// on the native [z][y][x] layout; each pass is the 1-D transform of every
// grid line, by a Felzenszwalb-Huttenlocher lower envelope of parabolas or,
// for short lines, by the direct minimum over the line (below).  Each thread owns one
// line: it gathers the line (stride 1, nx or nx*ny) into its own column of
// shared memory, builds the envelope there and writes the line back -- no
// transposition of the grid.  Envelope boundaries are exact fractions of
// integers, compared by 64-bit cross multiplication, so the result is the
// exact integer squared distance.
#include "ctx_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>

using namespace pm;

namespace {

constexpr int kEdtInf = 0x7fffffff;      // no site on the line (yet)
constexpr int kEdtMaxExtent = 1 << 14;

// A line of the pass: n elements base + i*se, base = a*sa + b*sb for line
// l = b*na + a.
struct EdtPass {
    int n, na, n_lines;
    long long sa, sb, se;
};

// Per-thread shared-memory columns of element i: f[i * T + t] (the line's
// values) and v[i * T + t] (the envelope's sites).  The envelope's
// boundaries are recomputed from neighbouring sites when needed, so a line
// costs 6 bytes of shared memory per element.
template <bool FROM_OCC>
__global__ void edt_pass_kernel(const void *in, int *out, EdtPass ps)
{
    extern __shared__ int s_edt[];
    const int T = blockDim.x, t = threadIdx.x;
    const int line = blockIdx.x * T + t;
    if (line >= ps.n_lines) return;
    const int n = ps.n;
    int *f = s_edt;                                               // [n][T] input values
    short *v = reinterpret_cast<short *>(s_edt + n * T);          // [n][T] sites
    const long long a = line % ps.na, b = line / ps.na;
    const long long base = a * ps.sa + b * ps.sb;

    // gather the line into this thread's column (8 loads in flight)
#pragma unroll 8
    for (int i = 0; i < n; ++i) {
        const long long idx = base + i * ps.se;
        int x;
        if (FROM_OCC) x = static_cast<const unsigned char *>(in)[idx] ? 0 : kEdtInf;
        else x = static_cast<const int *>(in)[idx];
        f[i * T + t] = x;
    }
    // Lower envelope of the parabolas y = (x - q)^2 + f[q] over the sites.
    // Parabolas u < w meet at s(u, w) = (h_w - h_u) / (2 (w - u)), h = f + q^2;
    // site v[k] covers [s(v[k-1], v[k]), s(v[k], v[k+1])).  The top two sites
    // stay in registers (vt, ht) and (vp, hp).
    int k = -1, vt = 0, vp = 0;
    long long ht = 0, hp = 0;
    for (int q = 0; q < n; ++q) {
        const int fq = f[q * T + t];
        if (fq == kEdtInf) continue;
        const long long hq = fq + static_cast<long long>(q) * q;
        // pop v[k] while s(v[k], q) <= s(v[k-1], v[k]), i.e.
        // (hq - ht) * 2 (vt - vp) <= (ht - hp) * 2 (q - vt)
        while (k >= 1 && (hq - ht) * (vt - vp) <= (ht - hp) * (q - vt)) {
            --k;
            vt = vp;
            ht = hp;
            if (k >= 1) {
                vp = v[(k - 1) * T + t];
                hp = f[vp * T + t] + static_cast<long long>(vp) * vp;
            }
        }
        ++k;
        v[k * T + t] = static_cast<short>(q);
        vp = vt;
        hp = ht;
        vt = q;
        ht = hq;
    }
    // evaluate the envelope at every element, advancing while the next
    // site's left boundary s(v[j], v[j+1]) lies below q
    int j = 0;
    int vj = k >= 0 ? v[t] : 0, vn = 0;
    long long hj = k >= 0 ? f[vj * T + t] + static_cast<long long>(vj) * vj : 0, hn = 0;
    if (k >= 1) {
        vn = v[T + t];
        hn = f[vn * T + t] + static_cast<long long>(vn) * vn;
    }
    for (int q = 0; q < n; ++q) {
        int d = kEdtInf;
        if (k >= 0) {
            while (j < k && hn - hj < 2LL * q * (vn - vj)) {   // s(vj, vn) < q
                ++j;
                vj = vn;
                hj = hn;
                if (j < k) {
                    vn = v[(j + 1) * T + t];
                    hn = f[vn * T + t] + static_cast<long long>(vn) * vn;
                }
            }
            d = static_cast<int>(hj - static_cast<long long>(vj) * vj) + (q - vj) * (q - vj);
        }
        out[base + q * ps.se] = d;
    }
}

// Shared memory per thread of a pass over lines of n elements (f, v and
// alignment slack).
size_t edt_bytes_per_thread(int n) { return static_cast<size_t>(n) * (4 + 2) + 4; }

// Threads per block: as many lines as fit 112 KiB of shared memory (two
// blocks per SM), a multiple of 32 when possible.
int edt_threads(int n)
{
    const size_t per = edt_bytes_per_thread(n);
    int T = static_cast<int>(std::min<size_t>(256, (112u << 10) / per));
    if (T >= 32) T -= T % 32;
    return std::max(T, 1);
}

template <bool FROM_OCC>
cudaError_t run_pass(const void *in, int *out, const EdtPass &ps, cudaStream_t s)
{
    const int T = edt_threads(ps.n);
    const size_t smem = edt_bytes_per_thread(ps.n) * T;
    cudaError_t e = cudaFuncSetAttribute(edt_pass_kernel<FROM_OCC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    edt_pass_kernel<FROM_OCC><<<(ps.n_lines + T - 1) / T, T, smem, s>>>(in, out, ps);
    return cudaGetLastError();
}

// Short lines (n <= kEdtBfMax) of the x and z passes take a direct pass
// instead of the envelope:
// a block stages 32 neighbouring lines as h_i = f_i + i^2 in shared memory,
// as floats, and every output d(x) = min_i (h_i - 2 x i) + x^2 is one FMA and
// one min per candidate i.  All values are integers below 2^24 (the caller
// checks the bound), so FP32 computes them exactly and the result equals
// the envelope's.  The work is O(n^2) per line against the envelope's O(n),
// but every (line, x) is independent, where the envelope walks its line
// with one thread.  Lines are staged along the line when it is contiguous
// and across lines otherwise, so loads and stores stay coalesced.
constexpr int kEdtBfMax = 256;
constexpr int kEdtBfLines = 32;
constexpr int kEdtBfPitch = kEdtBfLines + 1;   // shared-memory row pitch (no bank conflicts)
constexpr int kEdtBfWarps = 8;
constexpr int kEdtBfOut = 8;                   // outputs per thread per sweep over the candidates

__global__ void __launch_bounds__(kEdtBfWarps * 32)
edt_pass_direct_kernel(const int *in, int *out, EdtPass ps)
{
    extern __shared__ float s_bf[];
    const int n = ps.n;
    float *h = s_bf;                                                  // [n][pitch] h_i
    int *d = reinterpret_cast<int *>(s_bf + n * kEdtBfPitch);         // [n][pitch] outputs
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long line0 = static_cast<long long>(blockIdx.x) * kEdtBfLines;
    auto base_of = [&](long long l) { return (l % ps.na) * ps.sa + (l / ps.na) * ps.sb; };
    auto h_of = [&](long long idx, int i) -> float {
        const int x = in[idx];
        return x == kEdtInf ? CUDART_INF_F : static_cast<float>(x) + static_cast<float>(i * i);
    };
    if (ps.se == 1) {
        for (int li = warp; li < kEdtBfLines; li += kEdtBfWarps) {
            const long long l = line0 + li;
            const bool ok = l < ps.n_lines;
            const long long base = ok ? base_of(l) : 0;
            for (int i = lane; i < n; i += 32) h[i * kEdtBfPitch + li] = ok ? h_of(base + i, i) : CUDART_INF_F;
        }
    } else {
        const long long l = line0 + lane;
        const bool ok = l < ps.n_lines;
        const long long base = ok ? base_of(l) : 0;
        for (int i = warp; i < n; i += kEdtBfWarps)
            h[i * kEdtBfPitch + lane] = ok ? h_of(base + i * ps.se, i) : CUDART_INF_F;
    }
    __syncthreads();
    // lane: line; a warp takes kEdtBfOut consecutive outputs per sweep
    for (int x0 = warp * kEdtBfOut; x0 < n; x0 += kEdtBfWarps * kEdtBfOut) {
        float m[kEdtBfOut], c[kEdtBfOut];
#pragma unroll
        for (int k = 0; k < kEdtBfOut; ++k) {
            m[k] = CUDART_INF_F;
            c[k] = -2.0f * static_cast<float>(x0 + k);
        }
        float fi = 0.f;
#pragma unroll 4
        for (int i = 0; i < n; ++i) {
            const float hi = h[i * kEdtBfPitch + lane];
#pragma unroll
            for (int k = 0; k < kEdtBfOut; ++k) m[k] = fminf(m[k], fmaf(c[k], fi, hi));
            fi += 1.0f;
        }
#pragma unroll
        for (int k = 0; k < kEdtBfOut; ++k) {
            const int x = x0 + k;
            if (x < n)
                d[x * kEdtBfPitch + lane] =
                    m[k] == CUDART_INF_F ? kEdtInf : static_cast<int>(m[k] + static_cast<float>(x * x));
        }
    }
    __syncthreads();
    if (ps.se == 1) {
        for (int li = warp; li < kEdtBfLines; li += kEdtBfWarps) {
            const long long l = line0 + li;
            if (l >= ps.n_lines) continue;
            const long long base = base_of(l);
            for (int i = lane; i < n; i += 32) out[base + i] = d[i * kEdtBfPitch + li];
        }
    } else {
        const long long l = line0 + lane;
        if (l < ps.n_lines) {
            const long long base = base_of(l);
            for (int i = warp; i < n; i += kEdtBfWarps) out[base + i * ps.se] = d[i * kEdtBfPitch + lane];
        }
    }
}

// The first pass from occupancy, for lines up to kEdtBfMax: the squared
// distance along the line is to the nearest occupied element on either
// side, found by a forward and a backward sweep.  One thread per line (a
// warp takes 32 neighbouring lines, which sit next to each other in memory
// for the y pass, so the gathers are coalesced); the line's flags are
// staged in shared memory.
__global__ void __launch_bounds__(32)
edt_occ_sweep_kernel(const unsigned char *occ, int *out, EdtPass ps)
{
    extern __shared__ int s_sw[];                         // [n][pitch]: occupied, then the forward result
    const int n = ps.n, lane = threadIdx.x;
    const long long l = static_cast<long long>(blockIdx.x) * 32 + lane;
    if (l >= ps.n_lines) return;
    const long long base = (l % ps.na) * ps.sa + (l / ps.na) * ps.sb;
    int *c = s_sw + lane;
    // forward: distance to the nearest occupied element at or before i
    int last = -1;
    for (int i = 0; i < n; ++i) {
        const bool o = occ[base + i * ps.se] != 0;
        if (o) last = i;
        c[i * kEdtBfPitch] = last < 0 ? kEdtInf : (i - last) * (i - last);
    }
    // backward: the nearest at or after i, and the minimum of the two
    int next = -1;
    for (int i = n - 1; i >= 0; --i) {
        const int f = c[i * kEdtBfPitch];
        if (f == 0) next = i;
        const int b = next < 0 ? kEdtInf : (next - i) * (next - i);
        out[base + i * ps.se] = min(f, b);
    }
}

cudaError_t run_occ_sweep(const unsigned char *occ, int *out, const EdtPass &ps, cudaStream_t s)
{
    const size_t smem = static_cast<size_t>(ps.n) * kEdtBfPitch * sizeof(int);
    cudaError_t e = cudaFuncSetAttribute(edt_occ_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int blocks = static_cast<int>((ps.n_lines + 31) / 32);
    edt_occ_sweep_kernel<<<blocks, 32, smem, s>>>(occ, out, ps);
    return cudaGetLastError();
}

// The direct pass is exact when every staged value and every h_i - 2 x i
// stays below 2^24: inputs up to bound_in, plus at most 3 (n-1)^2.
bool direct_pass_exact(int n, long long bound_in)
{
    const long long m = n - 1;
    return n <= kEdtBfMax && bound_in + 3 * m * m < (1LL << 24);
}

cudaError_t run_direct_pass(const int *in, int *out, const EdtPass &ps, cudaStream_t s)
{
    const size_t smem = 2 * static_cast<size_t>(ps.n) * kEdtBfPitch * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(edt_pass_direct_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int blocks = static_cast<int>((ps.n_lines + kEdtBfLines - 1) / kEdtBfLines);
    edt_pass_direct_kernel<<<blocks, kEdtBfWarps * 32, smem, s>>>(in, out, ps);
    return cudaGetLastError();
}

// Squared EDT of occ [nz][ny][nx] into d2 (int32, kEdtInf without any site);
// tmp is scratch of the same size (y pass into d2, x pass into tmp, z pass
// back into d2).
cudaError_t edt3d(const unsigned char *occ, int nx, int ny, int nz, int *d2, int *tmp, cudaStream_t s)
{
    const long long sy = nx, sz = static_cast<long long>(nx) * ny;
    // y lines (x, z), x fastest across threads: coalesced gathers
    EdtPass py{ny, nx, nx * nz, 1, sz, sy};
    // x lines (y, z): each thread reads its own contiguous line
    EdtPass px{nx, ny, ny * nz, sy, sz, 1};
    // z lines (x, y): coalesced
    EdtPass pz{nz, nx, nx * ny, 1, sy, sz};
    // each pass direct when exact for its line length and input bound, else
    // the envelope
    const long long by = static_cast<long long>(ny - 1) * (ny - 1), bx = static_cast<long long>(nx - 1) * (nx - 1);
    cudaError_t e = ny <= kEdtBfMax ? run_occ_sweep(occ, d2, py, s) : run_pass<true>(occ, d2, py, s);
    if (e == cudaSuccess)
        e = direct_pass_exact(nx, by) ? run_direct_pass(d2, tmp, px, s) : run_pass<false>(d2, tmp, px, s);
    if (e == cudaSuccess)
        e = direct_pass_exact(nz, by + bx) ? run_direct_pass(tmp, d2, pz, s) : run_pass<false>(tmp, d2, pz, s);
    return e;
}

// phi = res sqrt(D) in metres, rounded once from FP64 to the storage type;
// without any occupied voxel phi = kFarField.
constexpr double kFarField = 1e10;

// The squared distances of a grid take at most (nx-1)^2 + (ny-1)^2 +
// (nz-1)^2 + 1 values; up to kPhiTableMax of them, a table of their metres,
// computed with the same FP64 expression, turns the conversion into a
// gather (FP64 is slow on this GPU).
constexpr size_t kPhiTableMax = size_t(1) << 22;

__global__ void phi_table_kernel(float *table, size_t n, double res)
{
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x)
        table[i] = static_cast<float>(res * sqrt(static_cast<double>(i)));
}

__device__ __forceinline__ void store_phi(void *phi, size_t i, float v, int dtype)
{
    if (dtype == PM_F32) static_cast<float *>(phi)[i] = v;
    else if (dtype == PM_F16) static_cast<__half *>(phi)[i] = __float2half_rn(v);
    else static_cast<__nv_bfloat16 *>(phi)[i] = __float2bfloat16_rn(v);
}

__global__ void d2_to_phi_table_kernel(const int *d2, void *phi, size_t n, const float *table, size_t table_n,
                                       double res, int dtype)
{
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const int d = d2[i];
        float v;
        if (d == kEdtInf) v = static_cast<float>(kFarField);
        else if (static_cast<size_t>(d) < table_n) v = __ldg(table + d);
        else v = static_cast<float>(res * sqrt(static_cast<double>(d)));   // not reached for a grid's own transform
        store_phi(phi, i, v, dtype);
    }
}

__global__ void d2_to_phi_kernel(const int *d2, void *phi, size_t n, double res, int dtype)
{
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const int d = d2[i];
        const double m = d == kEdtInf ? kFarField : res * sqrt(static_cast<double>(d));
        store_phi(phi, i, static_cast<float>(m), dtype);
    }
}

// Robot mask: the world centre and radius (+ inflate) of every sphere at
// configuration q, one thread per sphere; then blocks (s, z) clear the
// voxels of sphere s's bounding box, z-slices z, z + gridDim.y, ..., whose
// centres lie in the closed ball.
__global__ void sphere_world_kernel(const RobotConst rc, const float *q, float inflate, float4 *out)
{
    const int s = threadIdx.x;
    if (s >= rc.n_spheres) return;
    int link = 0;
    while (link < kNJ && rc.link_begin[link + 2] <= s) ++link;   // sphere s lies on frame link + 1
    Frame F = base_frame();
    for (int j = 0; j <= link; ++j) dh_step(F, rc.ca[j], rc.sa[j], rc.a[j], rc.d[j], q[j] + rc.th0[j], rc.poly);
    const f3 p = frame_point(F, rc.sph_off[s][0], rc.sph_off[s][1], rc.sph_off[s][2]);
    out[s] = make_float4(p.x, p.y, p.z, rc.sph_r[s] + inflate);
}

constexpr int kMaskSlices = 8;

__global__ void robot_mask_kernel(const float4 *spheres, unsigned char *occ, int nx, int ny, int nz, float res,
                                  float ox, float oy, float oz)
{
    const float4 c = spheres[blockIdx.x];
    const float r = c.w;
    // voxel index range whose centres can lie within r (one voxel of slack)
    const float lo[3] = {(c.x - r - ox) / res - 1.5f, (c.y - r - oy) / res - 1.5f, (c.z - r - oz) / res - 1.5f};
    const float hi[3] = {(c.x + r - ox) / res + 0.5f, (c.y + r - oy) / res + 0.5f, (c.z + r - oz) / res + 0.5f};
    const int n[3] = {nx, ny, nz};
    int b0[3], b1[3];
    for (int a = 0; a < 3; ++a) {
        b0[a] = static_cast<int>(fminf(fmaxf(floorf(lo[a]), 0.f), static_cast<float>(n[a])));
        b1[a] = static_cast<int>(fminf(fmaxf(ceilf(hi[a]), 0.f), static_cast<float>(n[a])));
    }
    const int bx = b1[0] - b0[0], by = b1[1] - b0[1];
    if (bx <= 0 || by <= 0) return;
    const int cnt = bx * by;
    const float r2 = r * r;
    for (int l = b0[2] + static_cast<int>(blockIdx.y); l < b1[2]; l += gridDim.y) {
        const float dz = fmaf(static_cast<float>(l) + 0.5f, res, oz) - c.z;
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            const int i = b0[0] + t % bx, j = b0[1] + t / bx;
            const float dx = fmaf(static_cast<float>(i) + 0.5f, res, ox) - c.x;
            const float dy = fmaf(static_cast<float>(j) + 0.5f, res, oy) - c.y;
            if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) <= r2) occ[(static_cast<size_t>(l) * ny + j) * nx + i] = 0;
        }
    }
}

pm_status map_err(pm_ctx *c, pm_status st, const char *msg)
{
    if (c) c->err = msg;
    return st;
}

} // namespace

extern "C" {

pm_status pm_edt_squared(const uint8_t *occ, int nx, int ny, int nz, int32_t *d2, void *cuda_stream)
{
    // extents up to 2^14 keep every squared distance, parabola height and
    // boundary numerator inside int32 and every site index in a short
    if (!occ || !d2 || nx < 1 || ny < 1 || nz < 1 || nx > kEdtMaxExtent || ny > kEdtMaxExtent ||
        nz > kEdtMaxExtent)
        return PM_EINVAL;
    const size_t n = static_cast<size_t>(nx) * ny * nz;
    if (n >= (1ull << 31)) return PM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int *tmp = nullptr;
    cudaError_t e = cudaMallocAsync(&tmp, n * sizeof(int), s);
    if (e == cudaSuccess) e = edt3d(occ, nx, ny, nz, d2, tmp, s);
    if (tmp) cudaFreeAsync(tmp, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? PM_ENOMEM : PM_ECUDA;
    }
    return PM_OK;
}

pm_status pm_robot_mask(pm_ctx *c, uint8_t *occ, const float *q, float inflate, void *cuda_stream)
{
    if (!c) return PM_EINVAL;
    if (!occ || !q) return map_err(c, PM_EINVAL, "NULL occupancy or configuration");
    if (!std::isfinite(inflate) || inflate < 0.f) return map_err(c, PM_EINVAL, "inflate must be finite and >= 0");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard dg(c->device);
    cudaStream_t s = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : c->stream;
    // q: host or device [7]
    cudaPointerAttributes pa{};
    const bool dq = cudaPointerGetAttributes(&pa, q) == cudaSuccess && pa.type == cudaMemoryTypeDevice;
    cudaGetLastError();
    const float *qd = q;
    if (!dq) {
        for (int j = 0; j < kNJ; ++j)
            if (!std::isfinite(q[j])) return map_err(c, PM_EINVAL, "q has a non-finite entry");
        float *slot = c->d_c0 + 32;            // the mask's slot of the context's small scratch
        if (cudaMemcpyAsync(slot, q, kNJ * sizeof(float), cudaMemcpyHostToDevice, s) != cudaSuccess) {
            cudaGetLastError();
            return map_err(c, PM_ECUDA, "copy of q failed");
        }
        qd = slot;
    }
    if (c->rc.n_spheres > 0) {
        if (!c->d_mask_spheres && cudaMalloc(&c->d_mask_spheres, kMaxSpheres * sizeof(float4)) != cudaSuccess) {
            cudaGetLastError();
            return map_err(c, PM_ENOMEM, "robot mask scratch allocation failed");
        }
        sphere_world_kernel<<<1, 64, 0, s>>>(c->rc, qd, inflate, c->d_mask_spheres);
        robot_mask_kernel<<<dim3(c->rc.n_spheres, kMaskSlices), 256, 0, s>>>(
            c->d_mask_spheres, occ, c->gd.nx, c->gd.ny, c->gd.nz, c->gd.res, c->gd.origin[0], c->gd.origin[1],
            c->gd.origin[2]);
        if (cudaGetLastError() != cudaSuccess) return map_err(c, PM_ECUDA, "robot mask launch failed");
    }
    if (!dq && cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return map_err(c, PM_ECUDA, "robot mask failed");
    }
    return PM_OK;
}

pm_status pm_map_update(pm_ctx *c, const uint8_t *occ, int occ_is_device, const float *q_mask, float inflate,
                        void *cuda_stream)
{
    if (!c) return PM_EINVAL;
    if (!occ) return map_err(c, PM_EINVAL, "occupancy is NULL");
    const size_t n = c->grid_elems;
    if (c->gd.nx > kEdtMaxExtent || c->gd.ny > kEdtMaxExtent || c->gd.nz > kEdtMaxExtent)
        return map_err(c, PM_EINVAL, "grid extent above 16384 for the transform");
    cudaStream_t s = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : c->stream;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        DeviceGuard dg(c->device);
        if (!c->d_map_occ) {
            cudaError_t e = cudaMalloc(&c->d_map_occ, n);
            if (e == cudaSuccess) e = cudaMalloc(&c->d_map_a, n * sizeof(int));
            if (e == cudaSuccess) e = cudaMalloc(&c->d_map_b, n * sizeof(int));
            const size_t nt = static_cast<size_t>(c->gd.nx - 1) * (c->gd.nx - 1) +
                              static_cast<size_t>(c->gd.ny - 1) * (c->gd.ny - 1) +
                              static_cast<size_t>(c->gd.nz - 1) * (c->gd.nz - 1) + 1;
            // the metres table is optional: without it the conversion takes the
            // per-voxel FP64 path
            if (e == cudaSuccess && nt <= kPhiTableMax) {
                if (cudaMalloc(&c->d_phi_table, nt * sizeof(float)) == cudaSuccess) {
                    c->phi_table_n = nt;
                    phi_table_kernel<<<static_cast<unsigned>(std::min<size_t>((nt + 255) / 256, 4u * c->n_sm)), 256, 0,
                                       s>>>(c->d_phi_table, nt, static_cast<double>(c->gd.res));
                    e = cudaGetLastError();
                } else {
                    c->d_phi_table = nullptr;
                    cudaGetLastError();
                }
            }
            if (e != cudaSuccess) {
                cudaGetLastError();
                return map_err(c, PM_ENOMEM, "mapping scratch allocation failed");
            }
        }
        if (cudaMemcpyAsync(c->d_map_occ, occ, n, occ_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            s) != cudaSuccess) {
            cudaGetLastError();
            return map_err(c, PM_ECUDA, "occupancy copy failed");
        }
    }
    if (q_mask) {
        const pm_status st = pm_robot_mask(c, c->d_map_occ, q_mask, inflate, s);
        if (st != PM_OK) return st;
    }
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard dg(c->device);
    cudaError_t e = edt3d(c->d_map_occ, c->gd.nx, c->gd.ny, c->gd.nz, c->d_map_a, c->d_map_b, s);
    if (e == cudaSuccess) {
        const unsigned blocks = static_cast<unsigned>(std::min<size_t>((n + 255) / 256, 8u * c->n_sm));
        if (c->d_phi_table)
            d2_to_phi_table_kernel<<<blocks, 256, 0, s>>>(c->d_map_a, c->d_grid, n, c->d_phi_table, c->phi_table_n,
                                                          static_cast<double>(c->gd.res), c->gd.dtype);
        else
            d2_to_phi_kernel<<<blocks, 256, 0, s>>>(c->d_map_a, c->d_grid, n, static_cast<double>(c->gd.res),
                                                    c->gd.dtype);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return map_err(c, PM_ECUDA, "distance transform failed");
    }
    return finish_distance_field(c, s);
}

} // extern "C"
