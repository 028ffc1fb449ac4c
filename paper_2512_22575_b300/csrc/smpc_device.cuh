// Device arithmetic of one SMPC iteration (ParaMaP, arXiv 2512.22575, Sec. IV).
//
// Everything here is FP32 except the integer Philox generator.  The pieces:
//   - Philox4x32-10 (Salmon et al., SC'11) and Box-Muller normals (Eq. 27);
//   - modified-DH forward kinematics kept as three rotation columns and a
//     translation, updated joint by joint (Eq. 6);
//   - trilinear lookup of the distance field phi (Eq. 17);
//   - the SE(3) pose error xi = log(T_g^{-1} T_ee) (Eqs. 11-15) with the
//     closed form V(theta)^{-1} = I - [w]x/2 + c(theta) [w]x^2,
//     c(theta) = (1 - (theta/2) cot(theta/2)) / theta^2;
//   - the tightened joint-limit violation of Eq. 21.
#pragma once

#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math_constants.h>

namespace pm {

constexpr int kNJ = 7;            // joints of the compiled kinematic chain
constexpr int kMaxSpheres = 64;
// zero entries after the sphere tables: a batch of spheres may read up to
// kSpherePad - 1 entries past a frame's last sphere (masked, never used)
constexpr int kSpherePad = 4;
constexpr int kMaxHorizon = 256;
constexpr int kMaxSelfGroups = (kNJ * (kNJ + 1)) / 2;   // frame pairs (a <= b) of the self-collision set
constexpr int kMaxSelfPairs = 4096;
constexpr int kSelfDense = 4;        // spheres per frame of a dense self-collision group

// Coefficients of the sin/cos and ln polynomials (gen_sincos_poly.py) as the
// kernels read them, from their parameters: the (sin, cos) pairs are the
// operands of packed FMAs, the ln coefficients the addends of scalar ones
// (an FMA takes a constant-bank addend, not an immediate one).
struct PolyConst {
    float2 sc[4];                 // (sin, cos) pairs, highest degree first
    float ln[4];                  // the atanh bracket, lowest degree first
};

// Arm + cost constants, passed by value as a kernel parameter (constant bank).
struct RobotConst {
    int n_spheres;
    int link_begin[kNJ + 2];      // spheres of frame i (1..n) are [link_begin[i], link_begin[i+1])
    float ca[kNJ], sa[kNJ];       // cos/sin of alpha_{i-1}
    float a[kNJ], d[kNJ], th0[kNJ];
    float flange_d;
    float q_lo[kNJ], q_hi[kNJ];   // tightened boxes of Eq. 21
    float qd_lo[kNJ], qd_hi[kNJ];
    float qdd_lo[kNJ], qdd_hi[kNJ];
    float sph_off[kMaxSpheres + kSpherePad][3];
    float sph_r[kMaxSpheres];
    // A frame whose spheres' offsets lie on one line through its origin,
    // o_s = lambda_s w (up to one float32 ulp of |w|), has link_line = 1: its
    // centres are t + lambda_s R w, three FMAs each in grid coordinates
    // (R link_wg, the direction in grid units, is formed once per frame).
    unsigned char link_line[kNJ];
    float link_w[kNJ][3];
    float link_wg[kNJ][3];        // link_w / res: the direction in grid units
    // sph_ls[s] = (lambda_s, skip threshold of sphere s).  A sphere whose
    // cell has all 8 corners above its threshold has d_act - (phi - r) < 0
    // for every point of the cell, even after FP32 rounding of the
    // interpolation: its collision term is exactly 0.  The threshold is
    // (d_act + r_s)(1 + 1e-6) + 1e-6, rounded up.
    float2 sph_ls[kMaxSpheres + kSpherePad];
    float Q[6], QH[6];
    float w_env, d_act, w_self;
    float w_q, w_qd, w_qdd, w_s, w_ns;
    float q_ref[kNJ];
    // Self-collision set S (Eq. 18), grouped by the frames (a <= b) of its
    // two spheres; n_self_groups = 0 switches the term off.  A group whose
    // frames' bounding-sphere centres are farther apart than
    // sqrt(grp_thr2) holds no pair closer than the sum of its radii, so
    // its violations are exactly 0 and it is skipped.
    int n_self_groups;
    unsigned char grp_fa[kMaxSelfGroups], grp_fb[kMaxSelfGroups];   // frame index - 1
    unsigned short grp_begin[kMaxSelfGroups + 1];                    // pairs of group g
    // 1: group g holds every pair of its two frames' spheres (at most
    // kSelfDense each), in (a, b) order, so it is evaluated as a dense block
    unsigned char grp_dense[kMaxSelfGroups];
    unsigned char self_frames;    // 1: the self slots use the frame layout (see self_slots)
    float grp_thr2[kMaxSelfGroups];
    float link_c[kNJ][3];         // bounding-sphere centre of frame j+1's spheres, in that frame
    float link_w2[kNJ];           // |link_w|^2 (the rotated direction's squared length)
    PolyConst poly;               // the sin/cos and ln coefficients
    // the forward kinematics' per-joint constants in 8-byte pairs (one
    // constant load each): (ca, sa), (a, d), (th0, link_wg[0]),
    // (link_wg[1], link_wg[2]) and the frame's spheres (link_begin[j+1],
    // link_begin[j+2])
    float2 fk_cs[kNJ], fk_ad[kNJ], fk_tw[kNJ], fk_ww[kNJ];
    int2 fk_be[kNJ];
    // The iteration kernels run the chain in grid units (the base frame at
    // the world origin's grid coordinate, lengths divided by the voxel
    // size), so a frame's origin is already the texture coordinate of the
    // skip bounds: fk_ad is (a, d) / res, and these are the other lengths
    float flange_dg;                                 // flange_d / res
    float sph_off_g[kMaxSpheres + kSpherePad][3];    // sph_off / res
    // joints (2p, 2p+1), p < 3, of the boxes of Eq. 21 and of q_ref
    float2 q_lo_pk[3], q_hi_pk[3], qd_lo_pk[3], qd_hi_pk[3], qdd_lo_pk[3], qdd_hi_pk[3], q_ref_pk[3];
    float link_lc[kNJ];           // frame layout: the bounding centre link_c = link_lc link_w
    // device [n], grouped and ordered by (a, b) within a group: x = bits of
    // the internal sphere indices a | b << 8, y = r_a + r_b, z = a squared
    // distance above which the pair is apart (its violation is exactly 0)
    const float4 *self_pairs;
};

// Per-lane shared-memory slots of the self-collision term.  Sphere layout:
// the world centres of the step's spheres, then of the frames' bounding
// spheres.  Frame layout (self_frames, every group dense and every frame
// in a group on a line, its bounding-sphere centre too): per frame j, its
// origin t and its rotated direction v = R w, 6 floats in grid units (the
// chain's own origin and R w / res); every sphere and bounding centre of the
// frame is t + lambda v.  The sphere layout keeps a
// slot's 32 lanes contiguous (slot s of a lane at s * 32); the frame layout
// keeps a lane's 6 floats of a frame contiguous (frame j of lane l at
// j * 192 + 6 l: t.x, t.y, v.x, v.y, t.z, v.z), read and written as three
// 8-byte pairs (a warp's 8-byte accesses at a 24-byte lane stride fall in
// distinct banks per half-warp).
constexpr int kSelfFrameSlots = 6;
__host__ __device__ constexpr int self_slots(int n_spheres, bool frames)
{
    return frames ? kSelfFrameSlots * kNJ : 3 * n_spheres + 3 * kNJ;
}

struct GridConst {
    const void *phi;              // [nz][ny][nx], x fastest; float, half or bf16
    const float *cmin;            // [nz][ny][nx]: skip bound of the cell with base voxel
                                  // (i, j, l): min of the field over the voxels
                                  // [i-1, i+1] x [j-1, j+1] x [l-1, l+1] (clamped at 0)
    // cmin of the (nx-1) x (ny-1) x (nz-1) cells as a point-sampled texture
    // (clamped addressing, unnormalised coordinates), fetched at the raw grid
    // coordinate: the texture unit's fixed-point rounding of a coordinate
    // may reach the next cell up, whose bound also covers this one.
    cudaTextureObject_t cmin_tex;
    int nx, ny, nz;
    float inv_res;
    float bx, by, bz;             // -origin / res - 1/2: grid coordinate g = p / res + b
    float mx, my, mz;             // n - 1 (clamp bound)
    float2 inv_res_pk, bxy;       // (inv_res, inv_res) and (bx, by), for packed operations
    float res;                    // voxel size: p = (g - b) res
    float2 mbxy;                  // -(bx, by) res
    float mbz;                    // -bz res
    unsigned *err;                // bounds-checked builds: the context's violation word (else null)
};

// ------------------------------------------------------------ bounds checks
// A library built with PM_BOUNDS_CHECK checks the index of every field
// gather, shared-memory slot and partial / cost / trace write of the
// iteration kernels against its extent.  A violation sets its bit in the
// context's word (GridConst::err) and the access is skipped (a read takes
// element 0 instead); nothing traps.  In the normal build the checks
// compile away.
constexpr unsigned kErrField = 1u, kErrTile = 2u, kErrStage = 4u, kErrBlock = 8u, kErrUbar = 16u,
                   kErrCosts = 32u, kErrPartial = 64u, kErrTrace = 128u, kErrSelf = 256u;

__device__ __forceinline__ bool pm_ok(bool in_bounds, unsigned code, const GridConst &g)
{
#ifdef PM_BOUNDS_CHECK
    if (!in_bounds) {
        if (g.err) atomicOr(g.err, code);
        return false;
    }
    return true;
#else
    (void)in_bounds; (void)code; (void)g;
    return true;
#endif
}

// index i of an array of n elements, or 0 (flagged) when out of range
__device__ __forceinline__ long long pm_idx(long long i, long long n, unsigned code, const GridConst &g)
{
    return pm_ok(i >= 0 && i < n, code, g) ? i : 0;
}

// The scalars of one launch: Philox key words, iteration index (the
// counter's last word), dt and 1/lambda.
struct CallScalars {
    uint32_t seed_lo, seed_hi, iter;
    float dt, inv_lambda;
};

// Per-call state as each block holds it in shared memory.
struct InstanceState {
    float q0[8], qd0[8];
    float Rg[9];                  // row-major R_g
    float tg[3];
    float sigma[8];
    CallScalars cs;               // filled only from a call's device block (CallInputs::dyn)
};

// Per-call scalars in device memory (a replayed graph's launches read them
// there, so one graph serves every call of its shape): floats
// [kDynSigma, +7) sigma, then dt, 1/lambda and the words seed_lo, seed_hi and
// iter0 (the iteration index of the call's first iteration).
constexpr int kDynSigma = 32, kDynDt = 40, kDynInvLambda = 41, kDynSeedLo = 42, kDynSeedHi = 43,
              kDynIter0 = 44, kDynFloats = 48;

// Per-call inputs: device pointers to q_0, qdot_0 [7] and the row-major goal
// pose [16]; sigma by value.  dyn: null, or the call's device block (sigma
// and the scalars are then read from it; see kDyn*).
struct CallInputs {
    const float *q0, *qd0, *Tg;
    float sigma[8];
    const float *dyn;
};

// Fill the shared-memory state from the call inputs (threads of one block).
// With in.dyn the call's scalars come from its device block, the iteration
// index as iter0 + cs.iter (cs: the launch's arguments).
__device__ __forceinline__ void load_state(const CallInputs &in, const CallScalars &cs, float *s_state)
{
    InstanceState &st = *reinterpret_cast<InstanceState *>(s_state);
    const int t = threadIdx.x;
    if (t < kNJ) {
        st.q0[t] = in.q0[t];
        st.qd0[t] = in.qd0[t];
        st.sigma[t] = in.dyn ? in.dyn[kDynSigma + t] : in.sigma[t];
    } else if (t >= 32 && t < 44) {
        const int i = t - 32, r = i >> 2, c = i & 3;   // rows 0-2 of T_goal
        if (c < 3) st.Rg[3 * r + c] = in.Tg[4 * r + c];
        else st.tg[r] = in.Tg[4 * r + 3];
    } else if (t == 64 && in.dyn) {
        st.cs.seed_lo = __float_as_uint(in.dyn[kDynSeedLo]);
        st.cs.seed_hi = __float_as_uint(in.dyn[kDynSeedHi]);
        st.cs.iter = __float_as_uint(in.dyn[kDynIter0]) + cs.iter;
        st.cs.dt = in.dyn[kDynDt];
        st.cs.inv_lambda = in.dyn[kDynInvLambda];
    }
}
constexpr int kStateFloats = sizeof(InstanceState) / sizeof(float);

// Programmatic dependent launch (sm_90 and later): let the next kernel in
// the stream be scheduled now, then wait until every predecessor this grid
// depends on has completed and its writes are visible.  Both are no-ops for
// a kernel launched without the programmatic-serialisation attribute.
__device__ __forceinline__ void grid_dependency_prologue()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Coefficients of gen_sincos_poly.py (host copies; the kernels take them
// from RobotConst::poly, in the parameter bank):
// (sin, cos) pairs, highest degree first, and the ln bracket, lowest first.
constexpr float2 kSinCosPoly[4] = {{2.724328624e-06f, 2.445699101e-05f}, {-1.984003320e-04f, -1.388753648e-03f},
                                   {8.333331905e-03f, 4.166664928e-02f}, {-1.666666716e-01f, -5.0e-01f}};
constexpr float kLnP0 = 3.333333433e-01f, kLnP1 = 2.000006735e-01f, kLnP2 = 1.427491456e-01f,
                kLnP3 = 1.167523712e-01f;
inline PolyConst poly_const()
{
    PolyConst p;
    for (int i = 0; i < 4; ++i) p.sc[i] = kSinCosPoly[i];
    p.ln[0] = kLnP0; p.ln[1] = kLnP1; p.ln[2] = kLnP2; p.ln[3] = kLnP3;
    return p;
}
constexpr float kRound = 12582912.0f;                  // 1.5 2^23: x + kRound rounds x to an integer

// sin and cos of (pi/2) n + r, |r| <= 1.01 pi/4, given r and the bits qb of
// a float whose low two bits are n mod 4: sin r and cos r by the odd and even
// polynomials of gen_sincos_poly.py (least-squares fits on Chebyshev nodes,
// within 0.9 ulp in float32 evaluation), their Horner steps paired in packed
// FP32 FMAs, then the quadrant applied by a swap and two sign flips.
__device__ __forceinline__ void sincos_quadrant(float r, unsigned qb, const PolyConst &pc, float &s, float &c)
{
    const float z = r * r;
    const float2 zz = make_float2(z, z);
    float2 p = __ffma2_rn(zz, pc.sc[0], pc.sc[1]);
    p = __ffma2_rn(zz, p, pc.sc[2]);
    p = __ffma2_rn(zz, p, pc.sc[3]);
    const float sr = fmaf(r * z, p.x, r);
    const float cr = fmaf(z, p.y, 1.0f);
    const bool odd = (qb & 1u) != 0u;
    const float sv = odd ? cr : sr, cv = odd ? sr : cr;
    s = __uint_as_float(__float_as_uint(sv) ^ ((qb << 30) & 0x80000000u));          // n mod 4 in {2, 3}
    c = __uint_as_float(__float_as_uint(cv) ^ (((qb + 1u) << 30) & 0x80000000u));   // n mod 4 in {1, 2}
}

// sin and cos of a joint angle x (Eq. 6).  Cody-Waite reduction by pi/2:
// n = rint(x 2/pi), taken from the low bits of x 2/pi + 1.5 2^23 (valid for
// |x| < 2^22 pi/2), r = x - n p1 - n p2 - n p3 with p1 + p2 + p3 = pi/2 in
// three float32 parts; with FMA the first step is exact (x - n p1 is a
// multiple of 2^-24 below 1 in magnitude).  Then sincos_quadrant.  Within 2
// ulps for |x| <= 64 and 2^-23 absolute up to 1e4; NaN for non-finite x.
__device__ __forceinline__ void joint_sincos(float x, float &s, float &c, const PolyConst &kc)
{
    constexpr float kTwoOverPi = 0.636619772367581343f;
    constexpr float kPio2Hi = 1.57079637050628662f;        // float32(pi/2)
    constexpr float kPio2Mid = -4.371138828673793e-8f;    // float32(pi/2 - kPio2Hi)
    constexpr float kPio2Lo = -1.7763568394002505e-15f;   // float32(pi/2 - kPio2Hi - kPio2Mid)
    const float t = fmaf(x, kTwoOverPi, kRound);
    const float n = t - kRound;
    float r = fmaf(-n, kPio2Hi, x);
    r = fmaf(-n, kPio2Mid, r);
    r = fmaf(-n, kPio2Lo, r);
    sincos_quadrant(r, __float_as_uint(t), kc, s, c);
}

// ------------------------------------------------------------------ Philox
// Philox4x32: per round two 32x32 -> 64 bit products, words permuted and
// xored with the key; the key is bumped by the Weyl constants each round.
__device__ __forceinline__ void philox4x32_10(uint32_t &x0, uint32_t &x1, uint32_t &x2,
                                              uint32_t &x3, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, x0), lo0 = 0xD2511F53u * x0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, x2), lo1 = 0xCD9E8D57u * x2;
        const uint32_t y0 = hi1 ^ x1 ^ k0;
        const uint32_t y2 = hi0 ^ x3 ^ k1;
        x0 = y0; x1 = lo1; x2 = y2; x3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Round keys of Philox4x32-10: (k0 + r W0, k1 + r W1) for rounds r < 10.
// A kernel that knows the key at launch takes them as parameters, so the
// rounds read them in place instead of bumping the key.
__host__ __device__ inline void philox_round_keys(uint32_t k0, uint32_t k1, uint2 (&rk)[10])
{
    for (int r = 0; r < 10; ++r) {
        rk[r].x = k0 + static_cast<uint32_t>(r) * 0x9E3779B9u;
        rk[r].y = k1 + static_cast<uint32_t>(r) * 0xBB67AE85u;
    }
}

// philox4x32_10 with the round keys given
__device__ __forceinline__ void philox4x32_10_rk(uint32_t &x0, uint32_t &x1, uint32_t &x2, uint32_t &x3,
                                                 const uint2 (&rk)[10])
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, x0), lo0 = 0xD2511F53u * x0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, x2), lo1 = 0xCD9E8D57u * x2;
        const uint32_t y0 = hi1 ^ x1 ^ rk[r].x;
        const uint32_t y2 = hi0 ^ x3 ^ rk[r].y;
        x0 = y0; x1 = lo1; x2 = y2; x3 = lo0;
    }
}

// u = ((x >> 9) + 0.5) 2^-23: a 23-bit integer plus one half fits the 24-bit
// significand, so u is exact in FP32 and strictly inside (0, 1).
__device__ __forceinline__ float word_to_uniform(uint32_t x)
{
    // (i + 1/2) 2^-23 = i 2^-23 + 2^-24, exact either way
    return fmaf(static_cast<float>(x >> 9), 1.1920928955078125e-7f, 5.9604644775390625e-8f);
}

// ln u for u in [2^-24, 1) (the Box-Muller radius).  u = 2^e m with m in
// [sqrt(1/2), sqrt(2)), split at the bits of sqrt(1/2) (the reduction of
// the classic float logarithms, e.g. Tang's); ln m = 2 atanh(s) with
// s = (m - 1)/(m + 1) = f/(2 + f), f = m - 1 exact, |s| <= 0.172, by
// 2s (1 + s^2 P(s^2)), P the fit of gen_sincos_poly.py; e ln 2 in two
// float32 parts.  Within 2 ulps (1.6 in emulation, plus the quotient's).
__device__ __forceinline__ float ln_unit(float u, const PolyConst &pc)
{
    constexpr float kLn2Hi = 0.693147182464599609f;        // float32(ln 2)
    constexpr float kLn2Lo = -1.9046542121259336e-09f;     // float32(ln 2 - kLn2Hi)
    const unsigned b = __float_as_uint(u);
    const int e = static_cast<int>(b - 0x3f3504f3u) >> 23;
    const float m = __uint_as_float(b - (static_cast<unsigned>(e) << 23));
    const float f = m - 1.0f;
    const float sq = __fdividef(f, 2.0f + f);               // 2 + f in [1.7, 2.5]: no special cases
    const float z = sq * sq;
    float p = fmaf(z, pc.ln[3], pc.ln[2]);
    p = fmaf(z, p, pc.ln[1]);
    p = fmaf(z, p, pc.ln[0]);
    const float s2 = sq + sq;
    const float ef = static_cast<float>(e);
    return fmaf(ef, kLn2Hi, fmaf(ef, kLn2Lo, fmaf(s2 * z, p, s2)));
}

// Two standard normals from two words (Eq. 27): radius sqrt(-2 ln u0),
// angle 2 pi u1 = (pi/2) t with t = 4 u1 in (0, 4) exact, so the reduction
// is exact too (n = rint(t), f = t - n in [-1/2, 1/2]) and the angle's
// sin and cos come from sincos_quadrant at r = (pi/2) f.
__device__ __forceinline__ void box_muller(uint32_t w0, uint32_t w1, float &z0, float &z1, const PolyConst &kc)
{
    constexpr float kPio2 = 1.57079637050628662f;
    const float u0 = word_to_uniform(w0);
    // v = -2 ln u0 lies in [1.2e-7, 33.3] (u0 in [2^-24, 1 - 2^-24]), so
    // v rsqrt(v) needs no special cases: within 3 ulp of sqrt(v)
    const float v = -2.0f * ln_unit(u0, kc);
    const float r = v * rsqrtf(v);
    // t = 4 u1 = 4 ((i + 1/2) 2^-23) = i 2^-21 + 2^-22
    const float t = fmaf(static_cast<float>(w1 >> 9), 4.76837158203125e-7f, 2.384185791015625e-7f);
    const float tq = t + kRound;
    float s, c;
    sincos_quadrant((t - (tq - kRound)) * kPio2, __float_as_uint(tq), kc, s, c);
    z0 = r * c;
    z1 = r * s;
}

// Standard normals z[0..7] of roll-out m, step k (counter (m, k, b, iter)).
// kc: the polynomial coefficients (RobotConst::poly, or a diagnostic's copy);
// rk: the key's round keys (philox_round_keys), or null to derive them.
__device__ __forceinline__ void step_normals(uint32_t seed_lo, uint32_t seed_hi, uint32_t iter,
                                             uint32_t m, uint32_t k, float z[8], const PolyConst &kc,
                                             const uint2 (*rk)[10] = nullptr)
{
#pragma unroll
    for (uint32_t b = 0; b < 2; ++b) {
        uint32_t x0 = m, x1 = k, x2 = b, x3 = iter;
        if (rk) philox4x32_10_rk(x0, x1, x2, x3, *rk);
        else philox4x32_10(x0, x1, x2, x3, seed_lo, seed_hi);
        box_muller(x0, x1, z[4 * b + 0], z[4 * b + 1], kc);
        box_muller(x2, x3, z[4 * b + 2], z[4 * b + 3], kc);
    }
}

// ------------------------------------------------------------------ vectors
struct f3 { float x, y, z; };

// The x and y components go through the packed FP32 units (__fmul2_rn,
// __ffma2_rn, __fadd2_rn: two IEEE operations in one instruction), z through
// the scalar ones; the results are those of three scalar operations.
__device__ __forceinline__ f3 mk(float x, float y, float z) { return f3{x, y, z}; }
__device__ __forceinline__ f3 scale(float a, f3 x)
{
    const float2 xy = __fmul2_rn(make_float2(a, a), make_float2(x.x, x.y));
    return f3{xy.x, xy.y, a * x.z};
}
// a*x + y
__device__ __forceinline__ f3 axpy(float a, f3 x, f3 y)
{
    const float2 xy = __ffma2_rn(make_float2(a, a), make_float2(x.x, x.y), make_float2(y.x, y.y));
    return f3{xy.x, xy.y, fmaf(a, x.z, y.z)};
}
__device__ __forceinline__ f3 sub(f3 a, f3 b)
{
    const float2 xy = __fadd2_rn(make_float2(a.x, a.y), make_float2(-b.x, -b.y));
    return f3{xy.x, xy.y, a.z - b.z};
}
__device__ __forceinline__ float dot(f3 a, f3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ f3 cross(f3 a, f3 b)
{
    return f3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// Frame as rotation columns c1, c2, c3 and origin t (world coordinates).
struct Frame { f3 c1, c2, c3, t; };

__device__ __forceinline__ Frame base_frame()
{
    return Frame{mk(1.f, 0.f, 0.f), mk(0.f, 1.f, 0.f), mk(0.f, 0.f, 1.f), mk(0.f, 0.f, 0.f)};
}

// T <- T RotX(alpha) TransX(a) RotZ(theta) TransZ(d)  (modified DH, Eq. 6).
// kc: the polynomial coefficients as the kernel holds them (RobotConst::poly).
__device__ __forceinline__ void dh_step(Frame &F, float ca, float sa, float a, float d, float theta,
                                        const PolyConst &kc)
{
    F.t = axpy(a, F.c1, F.t);                       // TransX(a); RotX keeps the x axis
    const f3 x2 = axpy(sa, F.c3, scale(ca, F.c2));  // RotX(alpha): y' = ca y + sa z
    const f3 x3 = axpy(-sa, F.c2, scale(ca, F.c3)); //              z' = -sa y + ca z
    float s, c;
    joint_sincos(theta, s, c, kc);
    const f3 y1 = axpy(s, x2, scale(c, F.c1));      // RotZ(theta): x'' = c x + s y'
    const f3 y2 = axpy(-s, F.c1, scale(c, x2));     //              y'' = -s x + c y'
    F.c1 = y1;
    F.c2 = y2;
    F.c3 = x3;
    F.t = axpy(d, x3, F.t);                         // TransZ(d)
}

// A point in grid units, in metres: (g - b) res.
__device__ __forceinline__ f3 grid_to_metres(const GridConst &g, f3 p)
{
    const float2 xy = __ffma2_rn(make_float2(p.x, p.y), make_float2(g.res, g.res), g.mbxy);
    return mk(xy.x, xy.y, fmaf(p.z, g.res, g.mbz));
}

// Point o given in frame F, in world coordinates: R o + t.
__device__ __forceinline__ f3 frame_point(const Frame &F, float ox, float oy, float oz)
{
    return axpy(oz, F.c3, axpy(oy, F.c2, axpy(ox, F.c1, F.t)));
}

// ------------------------------------------------------------ distance field
template <typename T> __device__ __forceinline__ float grid_load(const T *p);
template <> __device__ __forceinline__ float grid_load<float>(const float *p) { return __ldg(p); }
template <> __device__ __forceinline__ float grid_load<__half>(const __half *p)
{
    return __half2float(__ldg(p));
}
template <> __device__ __forceinline__ float grid_load<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    return __bfloat162float(__ldg(p));
}

// Clamp a grid coordinate into [0, n-1] and split it into a cell index in
// [0, n-2] and a fraction in [0, 1].
__device__ __forceinline__ int cell(float g, float gmax, int n, float &f)
{
    g = fminf(fmaxf(g, 0.0f), gmax);                // NaN maps to 0 (fmaxf)
    const int i = min(static_cast<int>(g), n - 2);  // g >= 0: truncation is floor
    f = g - static_cast<float>(i);
    return i;
}

// Cell of a point: base voxel offset and fractions (clamped, Eq. 17 lookup).
struct Cell { int base; float fx, fy, fz; };

// Cell of grid coordinates (gx, gy, gz) = p / res + b.
__device__ __forceinline__ Cell locate_grid(const GridConst &g, float gx, float gy, float gz)
{
    Cell c;
    const int ix = cell(gx, g.mx, g.nx, c.fx);
    const int iy = cell(gy, g.my, g.ny, c.fy);
    const int iz = cell(gz, g.mz, g.nz, c.fz);
    c.base = (iz * g.ny + iy) * g.nx + ix;
    return c;
}

__device__ __forceinline__ Cell locate(const GridConst &g, f3 p)
{
    return locate_grid(g, fmaf(p.x, g.inv_res, g.bx), fmaf(p.y, g.inv_res, g.by), fmaf(p.z, g.inv_res, g.bz));
}

// The 8 corner samples of a cell, in the order (x, y, z) = 000, 100, 010,
// 110, 001, 101, 011, 111.
template <typename T>
__device__ __forceinline__ void corners(const GridConst &g, int base, float v[8])
{
    const int sy = g.nx, sz = g.nx * g.ny;
    base = static_cast<int>(pm_idx(base, static_cast<long long>(sz) * g.nz - sz - sy - 1, kErrField, g));
    const T *b = static_cast<const T *>(g.phi) + base;
    v[0] = grid_load(b);          v[1] = grid_load(b + 1);
    v[2] = grid_load(b + sy);     v[3] = grid_load(b + sy + 1);
    v[4] = grid_load(b + sz);     v[5] = grid_load(b + sz + 1);
    v[6] = grid_load(b + sz + sy); v[7] = grid_load(b + sz + sy + 1);
}

// Trilinear interpolation in x, then y, then z.
__device__ __forceinline__ float interpolate(const float v[8], float fx, float fy, float fz)
{
    const float c00 = fmaf(fx, v[1] - v[0], v[0]), c10 = fmaf(fx, v[3] - v[2], v[2]);
    const float c01 = fmaf(fx, v[5] - v[4], v[4]), c11 = fmaf(fx, v[7] - v[6], v[6]);
    const float c0 = fmaf(fy, c10 - c00, c00), c1 = fmaf(fy, c11 - c01, c01);
    return fmaf(fz, c1 - c0, c0);
}

// phi(p): trilinear interpolation of the voxel-centre samples (Eq. 17).
template <typename T>
__device__ __forceinline__ float phi_trilinear(const GridConst &g, f3 p)
{
    const Cell c = locate(g, p);
    float v[8];
    corners<T>(g, c.base, v);
    return interpolate(v, c.fx, c.fy, c.fz);
}

// ----------------------------------------------------------------- SE(3)
// xi = [v; w] = log(T_g^{-1} T) for T = (F.c1 F.c2 F.c3 | t), Eqs. 11-15.
// Rg row-major, tg: goal pose.
__device__ __forceinline__ void pose_error(const float *Rg, const float *tg, f3 c1, f3 c2,
                                           f3 c3, f3 t, float xi[6])
{
    // columns of R_g (rows of R_g^T)
    const f3 g0 = mk(Rg[0], Rg[3], Rg[6]);
    const f3 g1 = mk(Rg[1], Rg[4], Rg[7]);
    const f3 g2 = mk(Rg[2], Rg[5], Rg[8]);
    // R_delta = R_g^T R,  t_delta = R_g^T (t - t_g)
    const float r00 = dot(g0, c1), r01 = dot(g0, c2), r02 = dot(g0, c3);
    const float r10 = dot(g1, c1), r11 = dot(g1, c2), r12 = dot(g1, c3);
    const float r20 = dot(g2, c1), r21 = dot(g2, c2), r22 = dot(g2, c3);
    const f3 dt = sub(t, mk(tg[0], tg[1], tg[2]));
    const f3 td = mk(dot(g0, dt), dot(g1, dt), dot(g2, dt));

    const f3 vee = mk(r21 - r12, r02 - r20, r10 - r01);  // 2 sin(th) a
    const float nv = sqrtf(dot(vee, vee));
    const float cth = 0.5f * (r00 + r11 + r22 - 1.0f);   // cos(th)
    const float th = atan2f(0.5f * nv, cth);
    // The small-angle series and the quotient forms (nv = 2 sin th lies in
    // [2e-4, 2] where the quotients are used, so __fdividef, 2 ulp, needs no
    // special cases) are both evaluated and selected, without a branch; only
    // the rare near-pi regime branches.
    //   w = k_w vee, k_w = th / nv, or 1/2 + th^2/12 below th = 1e-4;
    //   v = V(th)^{-1} t_delta, c(th) = (1 - (th/2) cot(th/2)) / th^2 with
    //   (th/2) cot(th/2) = th (1 + cos th) / (2 sin th) = th (1 + cth) / nv,
    //   or 1/12 + th^2/720 below th = 1e-2.
    const float th2 = th * th;
    const float kw = th < 1e-4f ? 0.5f + th2 * (1.0f / 12.0f) : __fdividef(th, nv);
    float cc = th < 1e-2f ? (1.0f / 12.0f) + th2 * (1.0f / 720.0f)
                          : __fdividef(1.0f - __fdividef(th * (1.0f + cth), nv), th2);
    f3 w = scale(kw, vee);
    if (th >= CUDART_PI_F - 0.05f) {
        // Near pi: (R + R^T)/2 = cos(th) I + (1 - cos(th)) a a^T; take the axis
        // from the column with the largest diagonal, the sign from vee.
        const float inv = 1.0f / (1.0f - cth);
        const float b00 = (r00 - cth) * inv, b11 = (r11 - cth) * inv, b22 = (r22 - cth) * inv;
        const float b01 = 0.5f * (r01 + r10) * inv, b02 = 0.5f * (r02 + r20) * inv;
        const float b12 = 0.5f * (r12 + r21) * inv;
        f3 ax;
        if (b00 >= b11 && b00 >= b22) {
            const float s = sqrtf(fmaxf(b00, 0.0f));
            ax = mk(s, b01 / s, b02 / s);
        } else if (b11 >= b22) {
            const float s = sqrtf(fmaxf(b11, 0.0f));
            ax = mk(b01 / s, s, b12 / s);
        } else {
            const float s = sqrtf(fmaxf(b22, 0.0f));
            ax = mk(b02 / s, b12 / s, s);
        }
        ax = scale(rsqrtf(dot(ax, ax)), ax);
        const float dv = dot(ax, vee);
        float sgn;
        if (dv != 0.0f) {
            sgn = dv > 0.0f ? 1.0f : -1.0f;
        } else {
            const float big = fabsf(ax.x) >= fabsf(ax.y) && fabsf(ax.x) >= fabsf(ax.z) ? ax.x
                              : (fabsf(ax.y) >= fabsf(ax.z) ? ax.y : ax.z);
            sgn = big >= 0.0f ? 1.0f : -1.0f;
        }
        w = scale(sgn * th, ax);
        const float h = 0.5f * th;
        float sh, ch;
        sincosf(h, &sh, &ch);
        cc = (1.0f - h * ch / sh) / th2;
    }
    const f3 wxt = cross(w, td);
    const f3 wwxt = cross(w, wxt);
    const f3 v = axpy(cc, wwxt, axpy(-0.5f, wxt, td));
    xi[0] = v.x; xi[1] = v.y; xi[2] = v.z;
    xi[3] = w.x; xi[4] = w.y; xi[5] = w.z;
}

// 1/2 xi^T diag(Q) xi  (Eqs. 16, 25).
__device__ __forceinline__ float quad_cost(const float xi[6], const float *Q)
{
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < 6; ++i) s = fmaf(Q[i] * xi[i], xi[i], s);
    return 0.5f * s;
}

// delta(x) of Eq. 21 on the tightened box [lo, hi] (lo < hi): x - hi above
// the box, x - lo below it, 0 inside, as x minus x clamped to the box (the
// same value, rounding included; NaN for NaN x).
__device__ __forceinline__ float limit_violation(float x, float lo, float hi)
{
    return x - fminf(fmaxf(x, lo), hi);
}

// limit_violation of two joints at once
__device__ __forceinline__ float2 limit_violation_pk(float2 x, float2 lo, float2 hi)
{
    const float2 cl = make_float2(fminf(fmaxf(x.x, lo.x), hi.x), fminf(fmaxf(x.y, lo.y), hi.y));
    return __fadd2_rn(x, make_float2(-cl.x, -cl.y));
}

// ------------------------------------------------------ compensated sums
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void kahan_add(float &sum, float &comp, float x)
{
    const float y = x - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

} // namespace pm
