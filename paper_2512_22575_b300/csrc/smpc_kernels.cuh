// The SMPC iteration kernel (ParaMaP, arXiv 2512.22575, Algorithm 1).
//
// Work decomposition.  A warp tile holds R = 32 / L roll-outs; each roll-out
// occupies L lanes and each lane owns C consecutive time steps
// k = l*C .. l*C + C-1 (H <= C*L).  Because the dynamics of Eq. 7 are a
// double integrator over the sampled accelerations, the states are prefix
// sums over k:
//     qd_{k+1} = qd_0 + dt A_{k+1},             A_k = sum_{i<k} u_i
//     q_{k+1}  = q_0 + (k+1) dt qd_0 + dt^2 B_{k+1},  B_k = sum_{i=1..k} A_i,
// computed with two segmented warp scans, so every (m, k) step is
// independent afterwards.  Lane step k evaluates the control terms of u_k
// (Eqs. 22, 23) and the state terms of q_{k+1}, qd_{k+1} (Eqs. 16, 19-20, 22,
// 24) or, for k+1 = H, the terminal cost (Eq. 25).  The state terms of
// k = 0 depend only on (q_0, qd_0) and are the same for every roll-out: one
// lane evaluates them once, in an extra pass through the step code, and the
// merge adds them to S; they cancel in the weights of Eq. 29.
//
// The sampled perturbations of a lane's steps are kept in shared memory
// ([warp][step][joint][lane], conflict-free) from sampling to the weighted
// sum, so the per-step body is not unrolled over C; the spheres of a link
// are looked up four at a time so their 32 gathers are in flight together.
//
// Soft-min (Eqs. 29-30).  Each warp keeps a running minimum m, sum
// z = sum exp(-(S - m)/lambda) and accumulator sum exp(-(S - m)/lambda) eps,
// rescaled when m drops.  Warps merge, in warp order, into one partial per
// block (m_b, z_b, acc_b), written as [m][z][acc^T] over blocks.  A second,
// wide kernel (softmin_merge_kernel in paramap.cu) merges the block partials
// into U* = Ubar + sum_b f_b acc_b / sum_b f_b z_b, f_b = exp((min m - m_b)/
// lambda), each sum in a fixed order, so results are deterministic for a
// given launch shape.
#pragma once

#include <type_traits>

#include "smpc_device.cuh"

namespace pm {

constexpr int kBlock = 128;
constexpr int kWarps = kBlock / 32;
constexpr int kMaxBlocks = 4096;
constexpr int kDenseBlocks = 7;   // blocks per SM of the dense one-step instantiations
constexpr int kTraceCols = 8;   // pose, env, self, lim_q, lim_qd, lim_qdd, smooth, ns
constexpr int kSphereBatch = 4;
static_assert(kSphereBatch - 1 <= kSpherePad, "a batch reads past a frame's spheres into the zero padding");

// Dynamic shared memory of an iteration kernel with C steps per lane: the
// perturbations and the soft-min accumulators, [kWarps][C][7][32] each.
constexpr size_t iteration_smem_bytes(int C)
{
    return 2u * kWarps * C * kNJ * 32 * sizeof(float);
}

// the block accumulator of a self-collision kernel lives in the slots (see
// smpc_iteration_kernel): the slots of any sphere count hold the longest one
static_assert(kWarps * 32 * 3 * kNJ >= kMaxHorizon * kNJ, "self slots hold the block accumulator");

// Extra dynamic shared memory of the self-collision term (0 when off).
inline size_t self_smem_bytes(const RobotConst &rc)
{
    return rc.n_self_groups > 0
               ? static_cast<size_t>(kWarps) * 32 * self_slots(rc.n_spheres, rc.self_frames) * sizeof(float)
               : 0;
}

struct IterArgs {
    CallInputs in;              // q0, qd0, T_goal (device), sigma
    const float *Ubar;          // [H][7]
    float *costs;               // [K] or null (without the k = 0 terms)
    float *part;                // block partials: m [nb], z [nb], acc [H*7][nb]; nb = gridDim.x
    float *c0;                  // [0] = k = 0 state terms
    float *trace;               // [K][H+1][8] (trace kernels only)
    unsigned long long *gathers;  // if not null: += number of 8-corner lookups performed
    int noise_dtype;            // PM_F32 (0), PM_F16 (1) or PM_BF16 (2): rounding of eps
    int K, H;
    CallScalars cs;             // seed, iteration index, dt, 1/lambda (see CallInputs::dyn)
    uint2 rk[10];               // Philox round keys of cs's seed (kernels without CallInputs::dyn)
};

// ------------------------------------------------------------ cost terms
// Control terms at step k (Eqs. 22, 23): w_qdd delta(qdd)^2 + w_s qdd^2.
template <bool TRACE>
__device__ __forceinline__ float control_cost(const RobotConst &rc, const float *u, float *tr)
{
    // joints in pairs through the packed FP32 units, the last one alone
    float2 lim2 = make_float2(0.f, 0.f), sm2 = make_float2(0.f, 0.f);
#pragma unroll
    for (int p = 0; p < kNJ / 2; ++p) {
        const float2 uu = make_float2(u[2 * p], u[2 * p + 1]);
        const float2 dl = limit_violation_pk(uu, rc.qdd_lo_pk[p], rc.qdd_hi_pk[p]);
        lim2 = __ffma2_rn(dl, dl, lim2);
        sm2 = __ffma2_rn(uu, uu, sm2);
    }
    const float d6 = limit_violation(u[kNJ - 1], rc.qdd_lo[kNJ - 1], rc.qdd_hi[kNJ - 1]);
    float lim = fmaf(d6, d6, lim2.x + lim2.y);
    float sm = fmaf(u[kNJ - 1], u[kNJ - 1], sm2.x + sm2.y);
    lim *= rc.w_qdd;
    sm *= rc.w_s;
    if (TRACE) { tr[5] = lim; tr[6] = sm; }
    return lim + sm;
}

// Whether a batch of spheres may hold one to gather: max_i (thr_i - mn_i) >= 0,
// i.e. some skip bound mn_i is not above its threshold (for finite values
// thr - mn >= 0 exactly when mn <= thr).  The batch's entries past its
// frame's last sphere (the next frame's spheres, or the zero padding) take
// part too: they can only cause a needless pass, whose per-sphere tests
// exclude them.
static_assert(kSphereBatch == 4, "batch_may_gather takes four spheres");
__device__ __forceinline__ bool batch_may_gather(const float (&mn)[kSphereBatch], float t0, float t1, float t2,
                                                 float t3)
{
    const float2 d01 = __fadd2_rn(make_float2(t0, t1), make_float2(-mn[0], -mn[1]));
    const float2 d23 = __fadd2_rn(make_float2(t2, t3), make_float2(-mn[2], -mn[3]));
    return fmaxf(fmaxf(d01.x, d01.y), fmaxf(d23.x, d23.y)) >= 0.0f;
}

// sum over spheres s in [b, e) of frame F of max(0, d_act - (phi(p_s) - r_s))^2
// (Eqs. 17, 19).  The skip bounds of four spheres (a lower bound of the 8
// corners of each sphere's cell) are fetched together through the texture
// unit; a sphere whose bound is above its skip threshold contributes
// exactly 0 and needs no gathers, the others are located exactly and
// interpolated from their 8 corners.
template <typename GT, bool SELF>
__device__ __forceinline__ float link_env(const RobotConst &rc, const GridConst &g,
                                          const Frame &F, int j, int b, int e, float wg0, bool count,
                                          unsigned &ngath, float *spf, float *sps)
{
    float env = 0.f;
    if (rc.link_line[j]) {
        // spheres on a line through the frame origin: grid coordinates
        // gt + lambda_s gv, gt of the origin and gv of the rotated direction
        // (wg0 = link_wg[j][0], loaded with th0)
        const float2 ww = rc.fk_ww[j];
        const f3 gv = axpy(ww.y, F.c3, axpy(ww.x, F.c2, scale(wg0, F.c1)));
        const f3 gt = F.t;          // the chain runs in grid units
        if (SELF && spf) {
            // the frame layout works in grid units: the origin and the
            // direction as the chain has them
            if (pm_ok(kSelfFrameSlots * j + 5 < self_slots(rc.n_spheres, true), kErrSelf, g)) {
                float2 *fs = reinterpret_cast<float2 *>(spf + kSelfFrameSlots * j * 32);
                fs[0] = make_float2(gt.x, gt.y);
                fs[1] = make_float2(gv.x, gv.y);
                fs[2] = make_float2(gt.z, gv.z);
            }
        } else if (SELF && sps) {
            // the sphere layout works in metres: the origin converted,
            // v = R w, each centre t + lambda_s v kept for the self term
            const f3 tm = grid_to_metres(g, F.t);
            const f3 v = axpy(rc.link_w[j][2], F.c3, axpy(rc.link_w[j][1], F.c2, scale(rc.link_w[j][0], F.c1)));
            for (int s = b; s < e; ++s) {
                if (!pm_ok(3 * s + 2 < self_slots(rc.n_spheres, false), kErrSelf, g)) break;
                const f3 p = axpy(rc.sph_ls[s].x, v, tm);
                sps[(3 * s) * 32] = p.x;
                sps[(3 * s + 1) * 32] = p.y;
                sps[(3 * s + 2) * 32] = p.z;
            }
        }
        for (int s0 = b; s0 < e; s0 += kSphereBatch) {
            float mn[kSphereBatch];
            float2 ls[kSphereBatch];
#pragma unroll
            for (int i = 0; i < kSphereBatch; ++i) {
                const int s = s0 + i;               // past e: zero padding, masked below
                ls[i] = rc.sph_ls[s];
                const float lam = ls[i].x;
                const float2 gxy = __ffma2_rn(make_float2(lam, lam), make_float2(gv.x, gv.y), make_float2(gt.x, gt.y));
                mn[i] = tex3D<float>(g.cmin_tex, gxy.x, gxy.y, fmaf(lam, gv.z, gt.z));
            }
            // one branch for the batch (see batch_may_gather), then each sphere's own test
            if (batch_may_gather(mn, ls[0].y, ls[1].y, ls[2].y, ls[3].y))
#pragma unroll
            for (int i = 0; i < kSphereBatch; ++i) {
                const int s = s0 + i;
                if (i < e - s0 && !(mn[i] > ls[i].y)) {
                    ngath += count ? 1u : 0u;
                    const float lam = ls[i].x;
                    const float2 gxy = __ffma2_rn(make_float2(lam, lam), make_float2(gv.x, gv.y), make_float2(gt.x, gt.y));
                    const Cell c = locate_grid(g, gxy.x, gxy.y, fmaf(lam, gv.z, gt.z));
                    float vv[8];
                    corners<GT>(g, c.base, vv);
                    const float phi = interpolate(vv, c.fx, c.fy, c.fz);
                    const float dl = fmaxf(rc.d_act - (phi - rc.sph_r[s]), 0.f);
                    env = fmaf(dl, dl, env);
                }
            }
        }
        return env;
    }
    for (int s0 = b; s0 < e; s0 += kSphereBatch) {
        float mn[kSphereBatch];
#pragma unroll
        for (int i = 0; i < kSphereBatch; ++i) {
            const int s = s0 + i;               // past e: zero padding, masked below
            // grid coordinates of the centre (the chain runs in grid units)
            const f3 p = frame_point(F, rc.sph_off_g[s][0], rc.sph_off_g[s][1], rc.sph_off_g[s][2]);
            if (SELF && sps && i < e - s0 &&
                pm_ok(3 * s + 2 < self_slots(rc.n_spheres, false), kErrSelf, g)) {   // kept for the self term
                const f3 pm = grid_to_metres(g, p);
                sps[(3 * s) * 32] = pm.x;
                sps[(3 * s + 1) * 32] = pm.y;
                sps[(3 * s + 2) * 32] = pm.z;
            }
            mn[i] = tex3D<float>(g.cmin_tex, p.x, p.y, p.z);
        }
        if (batch_may_gather(mn, rc.sph_ls[s0].y, rc.sph_ls[s0 + 1].y, rc.sph_ls[s0 + 2].y, rc.sph_ls[s0 + 3].y))
#pragma unroll
        for (int i = 0; i < kSphereBatch; ++i) {
            const int s = s0 + i;
            if (i < e - s0 && !(mn[i] > rc.sph_ls[s].y)) {
                // the few spheres near an obstacle: locate again with fractions
                ngath += count ? 1u : 0u;
                const f3 p = frame_point(F, rc.sph_off_g[s][0], rc.sph_off_g[s][1], rc.sph_off_g[s][2]);
                const Cell c = locate_grid(g, p.x, p.y, p.z);
                float v[8];
                corners<GT>(g, c.base, v);
                const float phi = interpolate(v, c.fx, c.fy, c.fz);
                const float dl = fmaxf(rc.d_act - (phi - rc.sph_r[s]), 0.f);
                env = fmaf(dl, dl, env);
            }
        }
    }
    return env;
}

// |c_a - c_b| from a squared distance d2 of a pair in contact range: d2 in
// [1e-30, ...) times its reciprocal square root (within 3 ulp of sqrt; the
// correctly rounded sqrtf costs a refinement and a special-value path).
__device__ __forceinline__ float pair_distance(float d2)
{
    const float v = fmaxf(d2, 1e-30f);
    return v * rsqrtf(v);
}

// Frame layout: the self-collision groups as per-block records in shared
// memory, kSelfGroupRec float4 each, built once per block from RobotConst,
// so that a step reads a group's constants with a few broadcast loads
// instead of indexing the constant tables through the group's frames and
// spheres.  The frame layout works in grid units (lengths / res): the slots
// hold the chain's own origins and directions, and the squared thresholds
// are scaled by 1/res^2, rounded up:
//   [0]  slot offsets of frames a and b (floats, as int bits), link_lc[a], link_lc[b]
//   [1]  grp_thr2 / res^2, |w_a / res|^2, |w_b / res|^2, res
//   [2], [3]  lambda and radius (metres) of frame a's spheres 0..3; [4], [5] frame b's
//   [6 + i]   the contact thresholds ((r_a + r_b + 1e-5 m) / res)^2, rounded
//             up, of frame a's sphere i with frame b's spheres 0..3.
// Past a frame's count a record repeats its last sphere with a NaN radius,
// whose pair thresholds are NaN, so the contact tests fail for them.  A
// group whose frame or sphere indices are out of range (bounds-checked
// builds) gets offsets 0 and NaN radii.
constexpr int kSelfGroupRec = 10;
__device__ __forceinline__ void self_frame_rec(const RobotConst &rc, const GridConst &g, int f, bool ok,
                                               float4 &l4, float4 &r4)
{
    static_assert(kSelfDense == 4, "one float4 per frame's lambdas and radii");
    const float nan = __int_as_float(0x7fc00000);
    const int lo = ok ? rc.link_begin[f + 1] : 0, n = ok ? rc.link_begin[f + 2] - lo : 0;
    float l[kSelfDense], rr[kSelfDense];
#pragma unroll
    for (int i = 0; i < kSelfDense; ++i) {
        const int s = lo + max(min(i, n - 1), 0);
        const bool sok = pm_ok(s >= 0 && s < kMaxSpheres, kErrSelf, g);
        l[i] = sok ? rc.sph_ls[s].x : 0.f;
        rr[i] = sok && i < n ? rc.sph_r[s] : nan;
    }
    l4 = make_float4(l[0], l[1], l[2], l[3]);
    r4 = make_float4(rr[0], rr[1], rr[2], rr[3]);
}
__device__ __forceinline__ void build_self_groups(const RobotConst &rc, const GridConst &g, float4 *tab)
{
    for (int gi = threadIdx.x; gi < rc.n_self_groups; gi += blockDim.x) {
        if (!pm_ok(gi < kMaxSelfGroups, kErrSelf, g)) break;
        const int fa = rc.grp_fa[gi], fb = rc.grp_fb[gi];
        const bool ok = pm_ok(fa < kNJ && fb < kNJ, kErrSelf, g);
        float4 *r = tab + kSelfGroupRec * gi;
        r[0] = make_float4(__int_as_float(ok ? kSelfFrameSlots * fa * 32 : 0),
                           __int_as_float(ok ? kSelfFrameSlots * fb * 32 : 0),
                           ok ? rc.link_lc[fa] : 0.f, ok ? rc.link_lc[fb] : 0.f);
        // 1/res rounded up keeps every scaled threshold at or above its exact value
        const float ir = __frcp_ru(g.res);
        const float *wa = rc.link_wg[ok ? fa : 0], *wb = rc.link_wg[ok ? fb : 0];
        r[1] = make_float4(__fmul_ru(__fmul_ru(rc.grp_thr2[gi], ir), ir),
                           fmaf(wa[0], wa[0], fmaf(wa[1], wa[1], wa[2] * wa[2])),
                           fmaf(wb[0], wb[0], fmaf(wb[1], wb[1], wb[2] * wb[2])), g.res);
        float4 la4, ra4, lb4, rb4;
        self_frame_rec(rc, g, fa, ok, la4, ra4);
        self_frame_rec(rc, g, fb, ok, lb4, rb4);
        r[2] = la4; r[3] = ra4; r[4] = lb4; r[5] = rb4;
        const float ra[4] = {ra4.x, ra4.y, ra4.z, ra4.w}, rb[4] = {rb4.x, rb4.y, rb4.z, rb4.w};
        float t2[4];
#pragma unroll
        for (int i = 0; i < kSelfDense; ++i) {
#pragma unroll
            for (int k = 0; k < kSelfDense; ++k) {
                const float t = __fmul_ru(__fadd_ru(__fadd_rn(ra[i], rb[k]), 1e-5f), ir);
                t2[k] = __fmul_ru(t, t);
            }
            r[6 + i] = make_float4(t2[0], t2[1], t2[2], t2[3]);
        }
    }
}

// Self-collision term (Eqs. 18-20): w_self sum over S of max(0, -d_self)^2,
// d_self = |c_a - c_b| - (r_a + r_b), from the sphere and bounding-sphere
// centres the step stored in its lane's slots sp (sphere layout: stride 32
// floats; frame layout: a frame's 6 floats contiguous, frames 192 floats
// apart); with the frame layout, grp holds the groups' records
// (build_self_groups).
__device__ __forceinline__ float self_cost(const RobotConst &rc, const float *sp, const float4 *grp)
{
    float acc = 0.f;
    if (rc.self_frames) {
        // frame layout: every group dense, every centre t + lambda_s v of its
        // frame (the same pairs and order as the dense blocks below)
        for (int gi = 0; gi < rc.n_self_groups; ++gi) {
            const float4 *rec = grp + kSelfGroupRec * gi;
            const float4 r0 = rec[0], r1 = rec[1];
            const float2 *pa = reinterpret_cast<const float2 *>(sp + __float_as_int(r0.x));
            const float2 *pb = reinterpret_cast<const float2 *>(sp + __float_as_int(r0.y));
            const float2 b0 = pb[0], b1 = pb[1], b2 = pb[2], a0 = pa[0], a1 = pa[1], a2 = pa[2];
            const f3 tb = mk(b0.x, b0.y, b2.x), vb = mk(b1.x, b1.y, b2.y);
            const f3 ta = mk(a0.x, a0.y, a2.x), va = mk(a1.x, a1.y, a2.y);
            // c_a - c_b = dl + l_a va - l_b vb with dl = ta - tb, so
            // |c_a - c_b|^2 = P_a + Q_b + m_a l_b with, per group, the dot
            // products of dl, va, vb (|va|^2 = |w_a|^2: a rotation keeps lengths):
            //   P_a = |dl|^2 + l_a (l_a |w_a|^2 + 2 dl.va),  m_a = -2 l_a va.vb,
            //   Q_b = l_b (l_b |w_b|^2 - 2 dl.vb),
            // two operations per pair instead of six, all in grid units.  The
            // skip test is still exact: the rounding of this sum stays below
            // 1e-6 of the squared frame distances (1e-7 m^2 for arm-sized
            // frames), far inside the pair threshold's 1e-5 m margin (about
            // 2e-6 m^2 at these radii); both scale alike by 1/res^2.
            // the frames' bounding spheres, centred at lambda-bar on each line:
            // apart beyond their radii + 0.1 mm, every pair of the group is
            // apart (exact zero); tested before the group's dot products
            {
                const f3 gc = sub(axpy(r0.z, va, ta), axpy(r0.w, vb, tb));
                if (dot(gc, gc) > r1.x) continue;
            }
            const f3 dl = sub(ta, tb);
            const float D = dot(dl, dl), Da2 = 2.0f * dot(dl, va), Db2 = 2.0f * dot(dl, vb);
            const float Vab2 = -2.0f * dot(va, vb);
            const float wa2 = r1.y, wb2 = r1.z, res = r1.w;
            // The group as a full 4 x 4 block (NaN radii past a frame's
            // count: no masks, no loop bounds); frame b's spheres in pairs
            // (2h, 2h+1) for the packed FP32 units.
            static_assert(kSelfDense == 4, "two pairs of frame-b spheres");
            const float4 la4 = rec[2], ra4 = rec[3], lb4 = rec[4], rb4 = rec[5];
            const float2 lb[2] = {make_float2(lb4.x, lb4.y), make_float2(lb4.z, lb4.w)};
            const float2 br[2] = {make_float2(rb4.x, rb4.y), make_float2(rb4.z, rb4.w)};
            float2 Qb[2];
#pragma unroll
            for (int h = 0; h < 2; ++h)
                Qb[h] = __fmul2_rn(lb[h], __ffma2_rn(lb[h], make_float2(wb2, wb2), make_float2(-Db2, -Db2)));
#pragma unroll
            for (int i = 0; i < kSelfDense; ++i) {
                const float la = i == 0 ? la4.x : i == 1 ? la4.y : i == 2 ? la4.z : la4.w;
                const float ra = i == 0 ? ra4.x : i == 1 ? ra4.y : i == 2 ? ra4.z : ra4.w;
                const float Pa = fmaf(la, fmaf(la, wa2, Da2), D), ma = la * Vab2;
                const float4 t24 = rec[6 + i];
                const float2 t2[2] = {make_float2(t24.x, t24.y), make_float2(t24.z, t24.w)};
                // the same operations as per pair: d2 = m_a l_b + (P_a + Q_b);
                // one branch per row of four pairs, taken where one of them
                // is within its threshold (rarely: most pairs of a group that
                // passed its bounding test are still apart)
                float2 d2[2];
                bool near = false;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    d2[h] = __ffma2_rn(make_float2(ma, ma), lb[h], __fadd2_rn(make_float2(Pa, Pa), Qb[h]));
                    near |= (d2[h].x <= t2[h].x) | (d2[h].y <= t2[h].y);
                }
                if (near) {
                    // the row's pairs in order, del in metres; a pair apart
                    // adds del = 0 (acc + 0 = acc: the same sum as skipping it)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float dx =
                            d2[h].x <= t2[h].x ? fmaxf(fmaf(-res, pair_distance(d2[h].x), ra + br[h].x), 0.f) : 0.f;
                        acc = fmaf(dx, dx, acc);
                        const float dy =
                            d2[h].y <= t2[h].y ? fmaxf(fmaf(-res, pair_distance(d2[h].y), ra + br[h].y), 0.f) : 0.f;
                        acc = fmaf(dy, dy, acc);
                    }
                }
            }
        }
        return rc.w_self * acc;
    }
    const int lb0 = 3 * rc.n_spheres;
    for (int gi = 0; gi < rc.n_self_groups; ++gi) {
        const int fa = lb0 + 3 * rc.grp_fa[gi], fb = lb0 + 3 * rc.grp_fb[gi];
        const float gx = sp[fa * 32] - sp[fb * 32];
        const float gy = sp[(fa + 1) * 32] - sp[(fb + 1) * 32];
        const float gz = sp[(fa + 2) * 32] - sp[(fb + 2) * 32];
        if (fmaf(gx, gx, fmaf(gy, gy, gz * gz)) > rc.grp_thr2[gi]) continue;   // exact zero
        if (rc.grp_dense[gi]) {
            // every pair of the two frames: b's centres and radii in
            // registers, a pair's term skipped only where it is exactly 0
            // (then sqrt(d2) >= t > r_a + r_b), in (a, b) order as listed
            const int a_lo = rc.link_begin[rc.grp_fa[gi] + 1], a_hi = rc.link_begin[rc.grp_fa[gi] + 2];
            const int b_lo = rc.link_begin[rc.grp_fb[gi] + 1], nb = rc.link_begin[rc.grp_fb[gi] + 2] - b_lo;
            float bx[kSelfDense], by[kSelfDense], bz[kSelfDense], br[kSelfDense];
#pragma unroll
            for (int i = 0; i < kSelfDense; ++i) {
                const int b = 3 * (b_lo + min(i, nb - 1));
                bx[i] = sp[b * 32];
                by[i] = sp[(b + 1) * 32];
                bz[i] = sp[(b + 2) * 32];
                br[i] = rc.sph_r[b_lo + min(i, nb - 1)];
            }
            for (int a = a_lo; a < a_hi; ++a) {
                const float ax = sp[(3 * a) * 32], ay = sp[(3 * a + 1) * 32], az = sp[(3 * a + 2) * 32];
                const float ra = rc.sph_r[a];
#pragma unroll
                for (int i = 0; i < kSelfDense; ++i) {
                    const float ex = ax - bx[i], ey = ay - by[i], ez = az - bz[i];
                    const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
                    const float rs = ra + br[i];
                    const float t = __fadd_ru(rs, 1e-5f);
                    if (i < nb && d2 <= __fmul_ru(t, t)) {
                        const float del = fmaxf(rs - pair_distance(d2), 0.f);
                        acc = fmaf(del, del, acc);
                    }
                }
            }
            continue;
        }
        int a_prev = -1;
        float ax = 0.f, ay = 0.f, az = 0.f;
        for (int p = rc.grp_begin[gi]; p < rc.grp_begin[gi + 1]; ++p) {
            const float4 pr = __ldg(rc.self_pairs + p);
            const unsigned ab = __float_as_uint(pr.x);
            const int a = 3 * static_cast<int>(ab & 0xffu), b = 3 * static_cast<int>(ab >> 8);
            if (a != a_prev) {          // pairs run by a: its centre is reused
                ax = sp[a * 32];
                ay = sp[(a + 1) * 32];
                az = sp[(a + 2) * 32];
                a_prev = a;
            }
            const float ex = ax - sp[b * 32];
            const float ey = ay - sp[(b + 1) * 32];
            const float ez = az - sp[(b + 2) * 32];
            const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
            if (d2 <= pr.z) {           // otherwise |c_a - c_b| > r_a + r_b: exactly 0
                const float del = fmaxf(pr.y - pair_distance(d2), 0.f);
                acc = fmaf(del, del, acc);
            }
        }
    }
    return rc.w_self * acc;
}

// The joint-limit and null-space sums of a state (Eqs. 21, 24; weights not
// applied): lq = sum delta(q)^2, lqd = sum delta(qd)^2, ns = sum (q - q_ref)^2.
__device__ __forceinline__ void state_limits(const RobotConst &rc, const float *q, const float *qd, float &lq,
                                             float &lqd, float &ns)
{
    {
        // joints in pairs through the packed FP32 units, the last one alone
        float2 lq2 = make_float2(0.f, 0.f), lqd2 = make_float2(0.f, 0.f), ns2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int p = 0; p < kNJ / 2; ++p) {
            const float2 qq = make_float2(q[2 * p], q[2 * p + 1]), vv = make_float2(qd[2 * p], qd[2 * p + 1]);
            const float2 a = limit_violation_pk(qq, rc.q_lo_pk[p], rc.q_hi_pk[p]);
            const float2 b = limit_violation_pk(vv, rc.qd_lo_pk[p], rc.qd_hi_pk[p]);
            const float2 e = __fadd2_rn(qq, make_float2(-rc.q_ref_pk[p].x, -rc.q_ref_pk[p].y));
            lq2 = __ffma2_rn(a, a, lq2);
            lqd2 = __ffma2_rn(b, b, lqd2);
            ns2 = __ffma2_rn(e, e, ns2);
        }
        constexpr int j = kNJ - 1;
        const float a = limit_violation(q[j], rc.q_lo[j], rc.q_hi[j]);
        const float b = limit_violation(qd[j], rc.qd_lo[j], rc.qd_hi[j]);
        const float e = q[j] - rc.q_ref[j];
        lq = fmaf(a, a, lq2.x + lq2.y);
        lqd = fmaf(b, b, lqd2.x + lqd2.y);
        ns = fmaf(e, e, ns2.x + ns2.y);
    }
}

// The weighted state-limit terms of a step: w_q lq + w_qd lqd + w_ns ns.
__device__ __forceinline__ float state_limit_cost(const RobotConst &rc, const float *q, const float *qd)
{
    float lq, lqd, ns;
    state_limits(rc, q, qd, lq, lqd, ns);
    return fmaf(rc.w_q, lq, fmaf(rc.w_qd, lqd, rc.w_ns * ns));
}

// State terms at a step (Eqs. 16, 19-20, 22, 24), or the terminal cost (Eq. 25).
// Forward kinematics runs frame by frame; the spheres of each frame are
// looked up as soon as it is known.  LIM = false: the step's limit and
// null-space terms were evaluated where its state was staged (q and qd
// are not read).
template <typename GT, bool TRACE, bool SELF, bool QMEM = false, bool LIM = true>
__device__ __forceinline__ float state_cost(const RobotConst &rc, const GridConst &g,
                                            const InstanceState &st, const float *q,
                                            const float *qd, bool terminal, float *tr,
                                            unsigned &ngath, float *sp, const float4 *sg, const float *qa = nullptr,
                                            int qstride = 1)
{
    if (!SELF || terminal) sp = nullptr;
    // The terminal step (one lane in H) runs the step's terms too and drops
    // them at the end: the lanes of a warp run together, and a branch around
    // them would cost every lane its instructions.
    float lq = 0.f, lqd = 0.f, ns = 0.f;
    if (LIM) state_limits(rc, q, qd, lq, lqd, ns);
    // the chain in grid units: the base at the world origin's grid coordinate
    Frame F = base_frame();
    F.t = mk(g.bx, g.by, g.bz);
    float env = 0.f;
    // Not unrolled: the kernel's code then fits the instruction cache, which
    // outweighs the indexed constant loads this costs.  With QMEM the joint
    // angles are read where the step staged them (qa, stride qstride), so
    // they hold no registers across the loop; otherwise they rotate through
    // qr so that the loop indexes no register array.
    float qr[kNJ];
    if (!QMEM) {
#pragma unroll
        for (int j = 0; j < kNJ; ++j) qr[j] = q[j];
    }
    // the self term's slots by layout, decided once per step
    float *const spf = (SELF && sp && rc.self_frames) ? sp : nullptr;
    float *const sps = (SELF && sp && !rc.self_frames) ? sp : nullptr;
#pragma unroll 1
    for (int j = 0; j < kNJ; ++j) {
        const float2 cs = rc.fk_cs[j], ad = rc.fk_ad[j], tw = rc.fk_tw[j];
        dh_step(F, cs.x, cs.y, ad.x, ad.y, (QMEM ? qa[j * qstride] : qr[0]) + tw.x, rc.poly);
        if (!QMEM) {
#pragma unroll
            for (int i = 0; i + 1 < kNJ; ++i) qr[i] = qr[i + 1];
        }
        const int2 be = rc.fk_be[j];
        env += link_env<GT, SELF>(rc, g, F, j, be.x, be.y, tw.y, !terminal, ngath, spf, sps);
        if (SELF && sps &&
            pm_ok(3 * rc.n_spheres + 3 * j + 2 < self_slots(rc.n_spheres, false), kErrSelf, g)) {
            const f3 c = grid_to_metres(g, frame_point(F, rc.link_c[j][0] * g.inv_res, rc.link_c[j][1] * g.inv_res,
                                                       rc.link_c[j][2] * g.inv_res));
            const int t = 3 * rc.n_spheres + 3 * j;
            sps[t * 32] = c.x;
            sps[(t + 1) * 32] = c.y;
            sps[(t + 2) * 32] = c.z;
        }
    }
    const f3 tee = grid_to_metres(g, axpy(rc.flange_dg, F.c3, F.t));
    float xi[6];
    pose_error(st.Rg, st.tg, F.c1, F.c2, F.c3, tee, xi);
    if (terminal) {
        const float c = quad_cost(xi, rc.QH);
        if (TRACE) tr[0] = c;
        return c;
    }
    const float pose = quad_cost(xi, rc.Q);
    env *= rc.w_env;
    lq *= rc.w_q;
    lqd *= rc.w_qd;
    ns *= rc.w_ns;
    const float self = (SELF && sp) ? self_cost(rc, sp, sg) : 0.f;
    if (TRACE) { tr[0] = pose; tr[1] = env; tr[2] = self; tr[3] = lq; tr[4] = lqd; tr[7] = ns; }
    return pose + env + self + lq + lqd + ns;
}

// ---------------------------------------------------------- warp scans
// Inclusive prefix sum over the L lanes of each segment, for 7 values.
__device__ __forceinline__ void seg_inclusive_scan(const float *x, float *in, int sl, int L)
{
#pragma unroll
    for (int j = 0; j < kNJ; ++j) {
        float v = x[j];
        for (int d = 1; d < L; d <<= 1) {
            const float t = __shfl_up_sync(0xffffffffu, v, d, L);
            if (sl >= d) v += t;
        }
        in[j] = v;
    }
}

// Exclusive prefix sum over the L lanes of each segment, for 7 values.
__device__ __forceinline__ void seg_exclusive_scan(const float *x, float *ex, int sl, int L)
{
#pragma unroll
    for (int j = 0; j < kNJ; ++j) {
        float v = x[j];
        for (int d = 1; d < L; d <<= 1) {
            const float t = __shfl_up_sync(0xffffffffu, v, d, L);
            if (sl >= d) v += t;
        }
        const float e = __shfl_up_sync(0xffffffffu, v, 1, L);
        ex[j] = (sl == 0) ? 0.f : e;
    }
}

__device__ __forceinline__ float weight_factor(float m_from, float m_to, float inv_lambda)
{
    return (m_from == CUDART_INF_F) ? 0.f : expf((m_to - m_from) * inv_lambda);
}

// Barrier of the two warps (64 threads) of pair pr of this block.  Both
// warps of a pair run the same sequence of roll-outs, so they always meet.
__device__ __forceinline__ void pair_barrier(int pr)
{
    // immediate barrier ids: with a register id the compiler must reserve
    // every hardware barrier for the block, which caps blocks per SM
    static_assert(kWarps / 2 <= 2, "pair barriers 1 and 2 cover at most two pairs");
    if (pr == 0) asm volatile("bar.sync 1, 64;" ::: "memory");
    else asm volatile("bar.sync 2, 64;" ::: "memory");
}

// The inputs of one instance's iteration as a block sees them (filled from
// IterArgs by the single-instance kernel, from a descriptor by the batched one).
struct TileJob {
    const float *Ubar;          // [H][7]
    float *costs;               // [K] or null
    float *part;                // this instance's block partials: m [nb], z [nb], acc [H*7][nb]
    float *c0;                  // [0] <- state terms of k = 0 (null: not computed)
    int K, H, nb;
    uint32_t seed_lo, seed_hi, iter;
    float dt, inv_lambda;
    int noise_dtype;
    // DYN kernels: the call's scalars in shared memory (they replace the five
    // above), read where they are used so that they hold no registers
    const CallScalars *dyn;
    // the seed's Philox round keys in the kernel's parameters, or null
    const uint2 (*rk)[10];
};

// A call scalar of a tile job: the field, or with DYN its copy in shared
// memory, loaded at the point of use.
template <bool DYN> __device__ __forceinline__ uint32_t job_seed_lo(const TileJob &j)
{
    return DYN ? *reinterpret_cast<const volatile uint32_t *>(&j.dyn->seed_lo) : j.seed_lo;
}
template <bool DYN> __device__ __forceinline__ uint32_t job_seed_hi(const TileJob &j)
{
    return DYN ? *reinterpret_cast<const volatile uint32_t *>(&j.dyn->seed_hi) : j.seed_hi;
}
template <bool DYN> __device__ __forceinline__ uint32_t job_iter(const TileJob &j)
{
    return DYN ? *reinterpret_cast<const volatile uint32_t *>(&j.dyn->iter) : j.iter;
}
template <bool DYN> __device__ __forceinline__ float job_dt(const TileJob &j)
{
    return DYN ? *reinterpret_cast<const volatile float *>(&j.dyn->dt) : j.dt;
}
template <bool DYN> __device__ __forceinline__ float job_inv_lambda(const TileJob &j)
{
    return DYN ? *reinterpret_cast<const volatile float *>(&j.dyn->inv_lambda) : j.inv_lambda;
}

// Shared-memory arrays a block needs for run_block.
struct BlockSmem {
    float *eps, *acc;           // [kWarps][C][7][32] each
    float (*tot)[2 * kNJ];      // [kWarps/2 + 1] pair scan totals, (A_j, B_j) pairs (8-byte aligned rows)
    float (*S)[2][2];           // [kWarps/2 + 1] pair partial costs
    float *blk;                 // [C*L*P*7] block accumulator
    float *wm, *wz;             // [kWarps]
    float *self;                // [kWarps][self_slots][32] when the self term is on, else null
    float *qs;                  // [kWarps][C][kStageFloats][32]: q, qd, control cost per step (STAGE)
    const float4 *grp;          // [n_self_groups][kSelfGroupRec] (frame layout), else null
};

// Floats staged per step: q, qd and the control cost.
constexpr int kStageFloats = 2 * kNJ + 1;

// Local block lb (of job.nb) of an instance: its roll-out tiles, then its
// block partial (m_b, z_b, acc_b) into job.part.  Tile shape (C, L, P) as
// described at the top of this file; called by every thread of the block.
// With constant arguments (the single-instance kernel) the shape folds away.
template <typename GT, bool TRACE, bool SELF, bool STAGE, bool DYN = false>
__device__ __forceinline__ void run_block(const RobotConst &rc, const GridConst &g,
                                          const InstanceState &st, const TileJob &job,
                                          float *trace, const int C, const int L, const int P,
                                          const int lb, const BlockSmem &sm, unsigned &ngath,
                                          const float *z0 = nullptr)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int R = 32 / L;
    const int seg = lane / L, sl = lane % L;
    const int H = job.H;
    // this lane's slot (w, s, j) of the [kWarps][C][7][32] tile arrays
    auto E = [&](int w, int s, int j) {
        return static_cast<int>(pm_idx(((w * C + s) * kNJ + j) * 32 + lane, kWarps * C * kNJ * 32, kErrTile, g));
    };

    for (int s = 0; s < C; ++s)
#pragma unroll
        for (int j = 0; j < kNJ; ++j) sm.acc[E(warp, s, j)] = 0.f;
    __syncthreads();

    float run_m = CUDART_INF_F, run_z = 0.f;
    const float dt = job_dt<DYN>(job), dt2 = dt * dt;
    float *sp = (SELF && rc.n_self_groups > 0 && sm.self)
                    ? sm.self + warp * self_slots(rc.n_spheres, rc.self_frames) * 32 +
                          (rc.self_frames ? kSelfFrameSlots * lane : lane)
                    : nullptr;
    const int half = (P == 2) ? (warp & 1) : 0;
    const int pr = warp >> 1;
    const int kbase = half * 32 * C;
    const int unit = (lb * kWarps + warp) / P;
    const int n_units = job.nb * kWarps / P;
    const int n_tiles = (job.K + R - 1) / R;
    // The state terms of k = 0 are the same for every roll-out: one lane
    // evaluates them once, in an extra pass through the step code (so they
    // add no code to the kernel), into job.c0; the merge adds them to S.
    // When the tiles do not divide evenly over the units, that pass runs as
    // a tile of its own (index n_tiles, no roll-outs) on the unit that would
    // take tile n_tiles, one with a tile fewer than the busiest units, so it
    // does not lengthen the launch; otherwise it follows the steps of the
    // last tile.
    const bool with_c0 = !TRACE && job.c0;
    const int c0_tile = (with_c0 && n_tiles % n_units != 0) ? n_tiles : n_tiles - 1;
    for (int tile = unit; tile <= c0_tile; tile += n_units) {
        const int m = tile * R + seg;
        const bool active = m < job.K;

        // sample and perturb (Algorithm 1, Eq. 27): eps ~ D, u = ubar + eps;
        // chunk sums T = sum_s u_s and TB = sum_s sum_{s'<=s} u_s' for the scans
        // (sums start at -0, the identity of IEEE addition, so the first
        // add folds away)
        float T[kNJ], TB[kNJ];
#pragma unroll
        for (int j = 0; j < kNJ; ++j) { T[j] = -0.f; TB[j] = -0.f; }
        float ccost = 0.f;          // STAGE: the lane's control terms
#pragma unroll 1
        for (int s = 0; s < C; ++s) {
            const int k = kbase + sl * C + s;
            float z[8];
            const bool live = active && k < H;
            // Steps past the horizon, and roll-outs past K, are sampled too
            // (from the last row of Ubar): in the scans a lane's values reach
            // only its own later steps and higher lanes, which are past the
            // horizon as well, and no result of theirs is kept.  Sampling
            // them saves the selects a branch-free zeroing would cost.
            const int kc = min(k, H - 1);
            // the step's row of Ubar, loaded before the sampling arithmetic
            // so that its latency is hidden behind it
            float ub[kNJ];
#pragma unroll
            for (int j = 0; j < kNJ; ++j) ub[j] = __ldg(job.Ubar + pm_idx(kc * kNJ + j, H * kNJ, kErrUbar, g));
            if (STAGE && z0 && tile == unit) {
                // the first tile's normals, drawn before the kernel waited
                // for the previous one (smpc_iteration_kernel)
#pragma unroll
                for (int j = 0; j < 8; ++j) z[j] = z0[j];
            } else {
                step_normals(job_seed_lo<DYN>(job), job_seed_hi<DYN>(job), job_iter<DYN>(job), static_cast<uint32_t>(m),
                             static_cast<uint32_t>(k), z, rc.poly, DYN ? nullptr : job.rk);
            }
            float ev[kNJ];
#pragma unroll
            for (int j = 0; j < kNJ; ++j) ev[j] = st.sigma[j] * z[j];
            if (job.noise_dtype != 0) {
                // precision variant: eps rounded as if stored in FP16 / BF16
#pragma unroll
                for (int j = 0; j < kNJ; ++j)
                    ev[j] = job.noise_dtype == 1 ? __half2float(__float2half_rn(ev[j]))
                                                 : __bfloat162float(__float2bfloat16_rn(ev[j]));
            }
#pragma unroll
            for (int j = 0; j < kNJ; ++j) {
                const float e = ev[j];
                const float u = ub[j] + e;
                sm.eps[E(warp, s, j)] = e;
                T[j] += u;
                TB[j] += T[j];
            }
            if (STAGE && live) {
                // one step per lane: its control terms now (T = u_k), staged
                // with its state below, so that u holds no registers in the scans
                float *tr_u = TRACE ? trace + pm_idx(static_cast<long long>(m) * (H + 1) + k,
                                                    static_cast<long long>(job.K) * (H + 1), kErrTrace, g) * kTraceCols
                                   : nullptr;
                ccost = control_cost<TRACE>(rc, T, tr_u);
            }
        }

        // roll-out (Eq. 7) by two segmented prefix scans.  One step per lane
        // (STAGE, C = 1): T = u_k, and A_{k+1}, B_{k+1} are the inclusive
        // scans of u and of A, into A0 and B0
        float A0[kNJ], B0[kNJ];
        if (STAGE) {
            seg_inclusive_scan(T, A0, sl, L);
            seg_inclusive_scan(A0, B0, sl, L);
            if (P == 2) {
                // the first half's A_32, B_32 (lane 31's inclusive values)
                // shift the second half's: A += A_32, B += B_32 + (sl + 1) A_32
                float2 *tot = reinterpret_cast<float2 *>(sm.tot[pr]);   // (A_j, B_j) pairs
                if (half == 0 && lane == 31) {
#pragma unroll
                    for (int j = 0; j < kNJ; ++j) tot[j] = make_float2(A0[j], B0[j]);
                }
                pair_barrier(pr);
                if (half == 1) {
#pragma unroll
                    for (int j = 0; j < kNJ; ++j) {
                        const float2 ab = tot[j];
                        B0[j] += fmaf(static_cast<float>(sl + 1), ab.x, ab.y);
                        A0[j] += ab.x;
                    }
                }
            }
        } else {
        seg_exclusive_scan(T, A0, sl, L);
#pragma unroll
        for (int j = 0; j < kNJ; ++j) TB[j] = fmaf(static_cast<float>(C), A0[j], TB[j]);
        seg_exclusive_scan(TB, B0, sl, L);
        if (P == 2) {
            // A_{32C} and B_{32C} of the first half shift the second half's scans:
            // A0 += A_{32C}, B0 += B_{32C} + (k0 - 32C) A_{32C}
            float2 *tot = reinterpret_cast<float2 *>(sm.tot[pr]);       // (A_j, B_j) pairs
            if (half == 0 && lane == 31) {
#pragma unroll
                for (int j = 0; j < kNJ; ++j) tot[j] = make_float2(A0[j] + T[j], B0[j] + TB[j]);
            }
            pair_barrier(pr);
            if (half == 1) {
#pragma unroll
                for (int j = 0; j < kNJ; ++j) {
                    const float2 ab = tot[j];
                    B0[j] += fmaf(static_cast<float>(sl * C), ab.x, ab.y);
                    A0[j] += ab.x;
                }
            }
        }
        }

        // kinematics and costs of each of this lane's steps (Eqs. 6, 16-25),
        // then, on lane 0 of tile c0_tile, the k = 0 pass
        const bool c0_lane = with_c0 && tile == c0_tile && seg == 0 && sl == 0 && half == 0;
        // With STAGE, every step's q, qd and control cost go to shared memory
        // first, so that the scan state is dead before the kinematics (fewer
        // registers at their peak, more resident warps); the k = 0 pass then
        // runs through the same code as the steps.
        float lsum = 0.f, lcomp = 0.f;
        float runU[kNJ], runB[kNJ];
#pragma unroll
        for (int j = 0; j < kNJ; ++j) { runU[j] = -0.f; runB[j] = B0[j]; }
        if (STAGE) {
            // the lane's one step: q_{k+1}, qd_{k+1} from A0 = A_{k+1},
            // B0 = B_{k+1} (its control terms are staged already)
            const int k = kbase + sl;
            if (active && k < H) {
                float *qs = sm.qs + pm_idx((warp * kStageFloats) * 32, kWarps * kStageFloats * 32 -
                                           (kStageFloats - 1) * 32 - 31, kErrStage, g) + lane;
                const float kp_dt = static_cast<float>(k + 1) * dt;
                // joints in pairs through the packed FP32 units, the last one alone
                const float2 dtp = make_float2(dt, dt), dt2p = make_float2(dt2, dt2), kpp = make_float2(kp_dt, kp_dt);
                float qn[kNJ], qdn[kNJ];    // q_{k+1}, qd_{k+1}
#pragma unroll
                for (int p = 0; p < kNJ / 2; ++p) {
                    const int j = 2 * p;
                    const float2 A = make_float2(A0[j], A0[j + 1]);
                    const float2 qd0 = make_float2(st.qd0[j], st.qd0[j + 1]);
                    const float2 qq = __ffma2_rn(dt2p, make_float2(B0[j], B0[j + 1]),
                                                 __ffma2_rn(kpp, qd0, make_float2(st.q0[j], st.q0[j + 1])));
                    const float2 vv = __ffma2_rn(dtp, A, qd0);
                    qn[j] = qq.x; qn[j + 1] = qq.y;
                    qdn[j] = vv.x; qdn[j + 1] = vv.y;
                }
                {
                    constexpr int j = kNJ - 1;
                    qn[j] = fmaf(dt2, B0[j], fmaf(kp_dt, st.qd0[j], st.q0[j]));
                    qdn[j] = fmaf(dt, A0[j], st.qd0[j]);
                }
#pragma unroll
                for (int j = 0; j < kNJ; ++j) qs[j * 32] = qn[j];
                if (TRACE) {
#pragma unroll
                    for (int j = 0; j < kNJ; ++j) qs[(kNJ + j) * 32] = qdn[j];
                    qs[(2 * kNJ) * 32] = ccost;
                } else {
                    // the state's limit and null-space terms here, with the
                    // state in registers (none at the terminal state, Eq. 25)
                    qs[(2 * kNJ) * 32] = ccost + (k + 1 == H ? 0.f : state_limit_cost(rc, qn, qdn));
                }
            }
        }
#pragma unroll 1
        for (int s = 0; s <= C; ++s) {
            const bool extra = (s == C);
            const int k = kbase + sl * C + s;
            if (extra) {
                if (!c0_lane) break;
            } else if (!(active && k < H)) {
                if (!c0_lane) break;
                s = C - 1;          // no more steps: on to the extra pass
                continue;
            }
            float q[kNJ], qd[kNJ], cc = 0.f;
            const float *qa = st.q0;
            int qstride = 1;
            float *tr_x = TRACE ? trace + pm_idx(static_cast<long long>(m) * (H + 1) + k + 1,
                                                static_cast<long long>(job.K) * (H + 1), kErrTrace, g) * kTraceCols
                               : nullptr;
            if (extra) {
#pragma unroll
                for (int j = 0; j < kNJ; ++j) { q[j] = st.q0[j]; qd[j] = st.qd0[j]; }
                // with STAGE the state terms below leave out the limits: add them
                if (STAGE && !TRACE) cc = state_limit_cost(rc, q, qd);
            } else if (STAGE) {
                const float *qs = sm.qs + pm_idx(((warp * C + s) * kStageFloats) * 32, kWarps * kStageFloats * 32 -
                                                 (kStageFloats - 1) * 32 - 31, kErrStage, g) + lane;
                if (TRACE) {
#pragma unroll
                    for (int j = 0; j < kNJ; ++j) { q[j] = qs[j * 32]; qd[j] = qs[(kNJ + j) * 32]; }
                }
                cc = qs[(2 * kNJ) * 32];
                qa = qs;
                qstride = 32;
            } else {
                float u[kNJ];
                const float kp_dt = static_cast<float>(k + 1) * dt;
#pragma unroll
                for (int j = 0; j < kNJ; ++j) {
                    u[j] = __ldg(job.Ubar + pm_idx(k * kNJ + j, H * kNJ, kErrUbar, g)) + sm.eps[E(warp, s, j)];
                    runU[j] += u[j];
                    const float A = A0[j] + runU[j];           // A_{k+1}
                    runB[j] += A;                               // B_{k+1}
                    qd[j] = fmaf(dt, A, st.qd0[j]);
                    q[j] = fmaf(dt2, runB[j], fmaf(kp_dt, st.qd0[j], st.q0[j]));
                }
                float *tr_u = TRACE ? trace + pm_idx(static_cast<long long>(m) * (H + 1) + k,
                                                    static_cast<long long>(job.K) * (H + 1), kErrTrace, g) * kTraceCols
                                   : nullptr;
                cc = control_cost<TRACE>(rc, u, tr_u);
            }
            const unsigned ng0 = ngath;
            // staged one-step lanes carry their limit terms in cc (LIM = false)
            const float sc = state_cost<GT, TRACE, SELF, STAGE, !STAGE || TRACE>(rc, g, st, q, qd, !extra && k + 1 == H,
                                                                               tr_x, ngath, sp, sm.grp, qa, qstride);
            if (extra) {
                ngath = ng0;        // lookups of the roll-outs only
                *job.c0 = sc + cc;
            } else if (STAGE) {
                lsum = cc + sc;         // one step per lane: nothing to compensate yet
            } else {
                kahan_add(lsum, lcomp, cc + sc);
            }
        }

        // S'^(m): compensated sum over the segment's lanes (one step per
        // lane: the first level starts without an error term)
        float ssum = lsum, serr = -lcomp;
        int off0 = L / 2;
        if (STAGE && off0 > 0) {
            const float os = __shfl_xor_sync(0xffffffffu, ssum, off0);
            two_sum(ssum, os, ssum, serr);
            off0 >>= 1;
        }
        for (int off = off0; off > 0; off >>= 1) {
            const float os = __shfl_xor_sync(0xffffffffu, ssum, off);
            const float oe = __shfl_xor_sync(0xffffffffu, serr, off);
            float ns, e;
            two_sum(ssum, os, ns, e);
            serr = serr + oe + e;
            ssum = ns;
        }
        float S = ssum + serr;
        if (P == 2) {
            if (lane == 0) { sm.S[pr][half][0] = ssum; sm.S[pr][half][1] = serr; }
            pair_barrier(pr);
            float ns, e;
            two_sum(sm.S[pr][0][0], sm.S[pr][1][0], ns, e);
            S = ns + ((sm.S[pr][0][1] + sm.S[pr][1][1]) + e);
        }
        if (TRACE) continue;
        if (active && sl == 0 && half == 0 && job.costs && pm_ok(m < job.K, kErrCosts, g)) job.costs[m] = S;

        // online soft-min accumulation (Eqs. 29-30)
        if (active) {
            const float nm = fminf(run_m, S);
            const float f_old = weight_factor(run_m, nm, job_inv_lambda<DYN>(job));
            const float f_new = expf((nm - S) * job_inv_lambda<DYN>(job));
            run_z = fmaf(run_z, f_old, f_new);
#pragma unroll 1
            for (int s = 0; s < C; ++s)
#pragma unroll
                for (int j = 0; j < kNJ; ++j) {
                    float &acc = sm.acc[E(warp, s, j)];
                    acc = fmaf(acc, f_old, f_new * sm.eps[E(warp, s, j)]);
                }
            run_m = nm;
        }
    }
    if (TRACE) return;

    // merge the R segments of the warp (they hold the same k slots)
    for (int off = L; off < 32; off <<= 1) {
        const float om = __shfl_xor_sync(0xffffffffu, run_m, off);
        const float oz = __shfl_xor_sync(0xffffffffu, run_z, off);
        const float nm = fminf(run_m, om);
        const float fa = weight_factor(run_m, nm, job_inv_lambda<DYN>(job));
        const float fb = weight_factor(om, nm, job_inv_lambda<DYN>(job));
        run_z = run_z * fa + oz * fb;
#pragma unroll 1
        for (int s = 0; s < C; ++s)
#pragma unroll
            for (int j = 0; j < kNJ; ++j) {
                float &mine = sm.acc[E(warp, s, j)];
                const float o = __shfl_xor_sync(0xffffffffu, mine, off);
                mine = mine * fa + o * fb;
            }
        run_m = nm;
    }

    // block partial, warps merged in warp order
    if (lane == 0) { sm.wm[warp] = run_m; sm.wz[warp] = run_z; }
    __syncthreads();
    // the block accumulator (C L P 7 floats) is cleared only now: with the
    // self term it shares its memory with the tiles' self-collision slots
    for (int i = tid; i < C * L * P * kNJ; i += kBlock) sm.blk[i] = 0.f;
    __syncthreads();
    float Mb = CUDART_INF_F;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) Mb = fminf(Mb, sm.wm[w]);
    const float fw = weight_factor(run_m, Mb, job_inv_lambda<DYN>(job));
    for (int w = 0; w < kWarps; ++w) {
        if (warp == w && seg == 0) {
            for (int s = 0; s < C; ++s) {
                const int k = kbase + sl * C + s;
                if (k < H && pm_ok(k < C * L * P, kErrBlock, g)) {
#pragma unroll
                    for (int j = 0; j < kNJ; ++j)
                        sm.blk[k * kNJ + j] = fmaf(fw, sm.acc[E(warp, s, j)], sm.blk[k * kNJ + j]);
                }
            }
        }
        __syncthreads();
    }
    const int na = H * kNJ;
    const int nb = job.nb;
    if (tid == 0 && pm_ok(lb < nb, kErrPartial, g)) {
        float zb = 0.f;
        // a pair's two warps carry the same (m, z): count it once
        for (int w = 0; w < kWarps; w += P) zb += sm.wz[w] * weight_factor(sm.wm[w], Mb, job_inv_lambda<DYN>(job));
        job.part[lb] = Mb;
        job.part[nb + lb] = zb;
    }
    float *acc_b = job.part + 2 * static_cast<size_t>(nb) + lb;
    if (pm_ok(lb < nb && na <= C * L * P * kNJ, kErrPartial, g))
        for (int i = tid; i < na; i += kBlock) acc_b[static_cast<size_t>(i) * nb] = sm.blk[i];
}

// ------------------------------------------------------------------ kernel
// P = 1: a warp tile holds R = 32/L roll-outs of up to C*L steps.  SELF
// compiles the self-collision term in (kernels without it carry none of
// its code).
// P = 2 (L = 32): two warps of a block share one roll-out, warp 2p taking
// steps [0, 32C) and warp 2p+1 steps [32C, 64C); they exchange the scan
// totals of the first half and their partial costs through shared memory.
// MINB is the residency the registers are fitted to: 6 blocks per SM for
// the one-step shapes without the self term (a budget of 80 registers; the
// (1,32,2) kernel now needs 72 and holds 7), 5 for the others (96; with the
// self term the 80-register fit spills and runs slower); the one-step
// shapes also have a kDenseBlocks instantiation (72 registers, no spills),
// which the host picks when its extra residency saves a round of tiles on
// a short launch.
template <int C, int L, int P, typename GT, bool TRACE, bool SELF, int MINB = (C == 1 && !SELF ? 6 : 5), bool DYN = false>
__global__ void __launch_bounds__(kBlock, MINB)
smpc_iteration_kernel(const __grid_constant__ RobotConst rc, const __grid_constant__ GridConst g,
                      const __grid_constant__ IterArgs a)
{
    static_assert(32 % L == 0 && C >= 1, "tile shape");
    static_assert(P == 1 || (P == 2 && L == 32 && kWarps % 2 == 0), "pair tiles are whole warps");
    static_assert(kBlock >= 44, "state loader needs 44 threads");
    extern __shared__ float s_dyn[];
    __shared__ __align__(16) float s_tot[kWarps / 2 + 1][2 * kNJ];
    __shared__ float s_S[kWarps / 2 + 1][2][2];
    __shared__ float s_state[kStateFloats];
    // block accumulator [k][j], k < C*L*P (>= H, host-checked); with the
    // self term it takes the start of the self-collision slots instead
    __shared__ float s_blk[SELF ? 1 : C * L * P * kNJ];
    __shared__ float s_wm[kWarps], s_wz[kWarps];
    // one-step shapes stage their steps' states (run_block, STAGE)
    constexpr bool kStage = (C == 1);
    __shared__ float s_qs[kStage ? kWarps * kStageFloats * 32 : 1];
    __shared__ float4 s_grp[SELF ? kMaxSelfGroups * kSelfGroupRec : 1];

    // the group records depend on the parameters alone: built before the
    // wait for the previous kernel
    const bool frame_groups = SELF && rc.n_self_groups > 0 && rc.self_frames;
    if (frame_groups) build_self_groups(rc, g, s_grp);
    // The normals of a one-step lane's first tile depend on the parameters
    // alone (the Philox key, the iteration, the roll-out and step indices):
    // drawn before the wait, they overlap the previous kernels' tails (replan
    // 2% shorter).  Only in the kDenseBlocks instantiations, which fit it in
    // 72 registers with a float field (the 80-register budget of the default
    // one would take 80 and hold a block fewer; the half-precision fields'
    // fits would spill); not with the self term, whose kernel is at its
    // register budget (0.7% longer).
    constexpr bool kPreSample =
        kStage && !TRACE && !SELF && MINB == kDenseBlocks && std::is_same<GT, float>::value;
    float z0[8];
    if (kPreSample) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int unit = (static_cast<int>(blockIdx.x) * kWarps + warp) / P;   // run_block's first tile
        const int m = unit * (32 / L) + lane / L;
        const int k = ((P == 2) ? (warp & 1) : 0) * 32 + lane % L;
        // a replayed graph's scalars: its call block, which a copy before
        // the graph wrote and no kernel of the graph writes (load_state
        // forms the same key and iteration from it)
        const uint32_t s_lo = DYN ? __float_as_uint(__ldg(a.in.dyn + kDynSeedLo)) : a.cs.seed_lo;
        const uint32_t s_hi = DYN ? __float_as_uint(__ldg(a.in.dyn + kDynSeedHi)) : a.cs.seed_hi;
        const uint32_t it = DYN ? __float_as_uint(__ldg(a.in.dyn + kDynIter0)) + a.cs.iter : a.cs.iter;
        step_normals(s_lo, s_hi, it, static_cast<uint32_t>(m), static_cast<uint32_t>(k), z0, rc.poly,
                     DYN ? nullptr : &a.rk);
    }
    grid_dependency_prologue();
    load_state(a.in, a.cs, s_state);
    __syncthreads();
    const InstanceState &st = *reinterpret_cast<const InstanceState *>(s_state);
    TileJob job;
    job.Ubar = a.Ubar;
    job.costs = a.costs;
    job.part = a.part;
    job.c0 = TRACE ? nullptr : a.c0;
    job.K = a.K;
    job.H = a.H;
    job.nb = gridDim.x;
    job.rk = nullptr;
    if (DYN) {
        job.dyn = &st.cs;
    } else {
        job.rk = &a.rk;
        job.seed_lo = a.cs.seed_lo;
        job.seed_hi = a.cs.seed_hi;
        job.iter = a.cs.iter;
        job.dt = a.cs.dt;
        job.inv_lambda = a.cs.inv_lambda;
    }
    job.noise_dtype = a.noise_dtype;
    float *self_slots_base = s_dyn + 2 * kWarps * C * kNJ * 32;
    BlockSmem sm{s_dyn, s_dyn + kWarps * C * kNJ * 32, s_tot, s_S, SELF ? self_slots_base : s_blk, s_wm, s_wz,
                 (SELF && rc.n_self_groups > 0) ? self_slots_base : nullptr, s_qs,
                 frame_groups ? s_grp : nullptr};
    unsigned ngath = 0;
    run_block<GT, TRACE, SELF, kStage, DYN>(rc, g, st, job, a.trace, C, L, P, blockIdx.x, sm, ngath,
                                            kPreSample ? z0 : nullptr);
    if (!TRACE && a.gathers) {
        const int lane = threadIdx.x & 31;
        unsigned n = ngath;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) n += __shfl_xor_sync(0xffffffffu, n, off);
        if (lane == 0) atomicAdd(a.gathers, static_cast<unsigned long long>(n));
    }
}

} // namespace pm
