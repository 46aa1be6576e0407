// EWA projection of 3D Gaussians to 2D splats (forward and backward).
//
// One thread per (view, Gaussian) item.  Parameters are read from the SoA
// layout P[14][stride], so the 14 loads of a warp are each one coalesced
// 128-byte transaction.  The forward writes each item's splat record (one
// 64-byte line: u, v, conic, colour, opacity, the culling box, the tile test's
// bound, the depth and the radius; SplatRec) and its placement record (the
// tile rectangle, the listed tiles and the depth in 16 bytes), and adds the
// item to the pair count of each listed tile.  The
// backward recomputes the forward state from the parameters (cheaper than
// storing it) and sums the per-view contributions of a Gaussian in
// registers, so the parameter gradient is written once, without atomics: the
// view-independent state (rotation, 3D covariance, opacity) is built once per
// Gaussian, and since the scale and rotation gradients are linear in
// dL/dSigma, that is summed over the views and taken through the
// covariance's factorisation once.
//
// Sec. 4.4 fine-tunes "as in" 3D Gaussian Splatting; the constants are that
// method's (vbm_internal.h), except that the splat radius is the extent of the
// region where o e^power >= 1/255 (at most 3 sigma): every pixel outside it
// would skip the splat, so the image is the same with fewer (tile, splat)
// pairs.
#include "vbm_internal.h"

namespace vbm {
namespace {

struct ProjState {
    float mu[3], s[3], qn[4], qnorm, R[3][3], Sig[3][3];
    float t[3], itz, xz, yz, xzc, yzc;
    bool clampx, clampy, culled;
    float T0[3], T1[3];
    float a, b, c, det, opac;
};

__device__ __forceinline__ float clampf(float x, float lo, float hi) { return fminf(fmaxf(x, lo), hi); }

// The view-independent part: mean, scales, normalised quaternion, rotation,
// 3D covariance and opacity.
__device__ __forceinline__ void project_base(const float *__restrict__ P, int64_t stride, int64_t g, ProjState &st)
{
#pragma unroll
    for (int k = 0; k < 3; k++) st.mu[k] = P[k * stride + g];
#pragma unroll
    for (int k = 0; k < 3; k++) st.s[k] = expf(P[(3 + k) * stride + g]);
    float q[4];
#pragma unroll
    for (int k = 0; k < 4; k++) q[k] = P[(6 + k) * stride + g];
    st.qnorm = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    float inv = 1.0f / st.qnorm;
#pragma unroll
    for (int k = 0; k < 4; k++) st.qn[k] = q[k] * inv;
    float w = st.qn[0], x = st.qn[1], y = st.qn[2], z = st.qn[3];
    st.R[0][0] = 1.f - 2.f * (y * y + z * z); st.R[0][1] = 2.f * (x * y - w * z); st.R[0][2] = 2.f * (x * z + w * y);
    st.R[1][0] = 2.f * (x * y + w * z); st.R[1][1] = 1.f - 2.f * (x * x + z * z); st.R[1][2] = 2.f * (y * z - w * x);
    st.R[2][0] = 2.f * (x * z - w * y); st.R[2][1] = 2.f * (y * z + w * x); st.R[2][2] = 1.f - 2.f * (x * x + y * y);
    float s2[3] = {st.s[0] * st.s[0], st.s[1] * st.s[1], st.s[2] * st.s[2]};
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++)
            st.Sig[a][b] = st.R[a][0] * s2[0] * st.R[b][0] + st.R[a][1] * s2[1] * st.R[b][1] +
                           st.R[a][2] * s2[2] * st.R[b][2];
    st.opac = 1.0f / (1.0f + expf(-P[10 * stride + g]));
}

// The view-dependent part, from the base state: camera-space mean, culling,
// frustum clamp, the Jacobian rows T0, T1 (J W) and the 2D covariance.
__device__ __forceinline__ void project_view(const vbm_camera &cam, ProjState &st)
{
    const float *Wm = cam.R;
#pragma unroll
    for (int r = 0; r < 3; r++)
        st.t[r] = Wm[3 * r] * st.mu[0] + Wm[3 * r + 1] * st.mu[1] + Wm[3 * r + 2] * st.mu[2] + cam.t[r];
    st.culled = !(st.t[2] > cam.znear);
    st.clampx = st.clampy = false;
    if (st.culled) return;
    // one reciprocal of the depth and of each focal length instead of ten
    // divisions (their results differ by an ulp or so)
    const float itz = 1.0f / st.t[2], ifx = 1.0f / cam.fx, ify = 1.0f / cam.fy;
    st.itz = itz;
    st.xz = st.t[0] * itz;
    st.yz = st.t[1] * itz;
    float Wi = (float)cam.width, Hi = (float)cam.height;
    float xlo = (-kFrustumGuard * Wi - cam.cx) * ifx, xhi = ((1.f + kFrustumGuard) * Wi - cam.cx) * ifx;
    float ylo = (-kFrustumGuard * Hi - cam.cy) * ify, yhi = ((1.f + kFrustumGuard) * Hi - cam.cy) * ify;
    st.xzc = clampf(st.xz, xlo, xhi);
    st.yzc = clampf(st.yz, ylo, yhi);
    st.clampx = st.xzc != st.xz;
    st.clampy = st.yzc != st.yz;
    float J00 = cam.fx * itz, J02 = -cam.fx * st.xzc * itz;
    float J11 = cam.fy * itz, J12 = -cam.fy * st.yzc * itz;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        st.T0[k] = J00 * Wm[k] + J02 * Wm[6 + k];
        st.T1[k] = J11 * Wm[3 + k] + J12 * Wm[6 + k];
    }
    float ST0[3], ST1[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        ST0[i] = st.Sig[i][0] * st.T0[0] + st.Sig[i][1] * st.T0[1] + st.Sig[i][2] * st.T0[2];
        ST1[i] = st.Sig[i][0] * st.T1[0] + st.Sig[i][1] * st.T1[1] + st.Sig[i][2] * st.T1[2];
    }
    st.a = st.T0[0] * ST0[0] + st.T0[1] * ST0[1] + st.T0[2] * ST0[2] + kDilation;
    st.b = st.T0[0] * ST1[0] + st.T0[1] * ST1[1] + st.T0[2] * ST1[2];
    st.c = st.T1[0] * ST1[0] + st.T1[1] * ST1[1] + st.T1[2] * ST1[2] + kDilation;
    st.det = st.a * st.c - st.b * st.b;
    if (!(st.det > 0.f)) st.culled = true;
}

// Views [vb + blockIdx.y vpt, + vpt) of the call (clipped to vb + vc), one
// Gaussian per thread: the view-independent state (rotation, 3D covariance,
// opacity) is built once and projected for each of those views.  With
// several scenes vpt is 1 (consecutive views may render different scenes).
// Four resident blocks (64 registers): the kernel waits on its parameter and
// camera loads, and 32 warps per SM hide more of that than 24.
template <bool MULTI>
__global__ void __launch_bounds__(256, 4)
    k_preprocess_fwd(const float *__restrict__ P, int64_t stride, const vbm_camera *__restrict__ cams,
                                 const int64_t *__restrict__ scene_offset, const int32_t *__restrict__ view_scene,
                                 const int64_t *__restrict__ view_item_offset, int vb, int vc, int vpt, int TX,
                                 int TY, int tw, int th, int W, int H, SplatRec *__restrict__ rec,
                                 float4 *__restrict__ gs, uint4 *__restrict__ place,
                                 uint32_t *__restrict__ tile_count, uint32_t *__restrict__ touched)
{
    const int v_begin = vb + blockIdx.y * (MULTI ? vpt : 1);
    const int v_end = MULTI ? min(v_begin + vpt, vb + vc) : v_begin + 1;
    const int scene = view_scene ? view_scene[v_begin] : 0;
    const int64_t g0 = scene_offset[scene];
    const int64_t ns = scene_offset[scene + 1] - g0;
    const int64_t gl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = gl < ns;        // every lane stays for the warp-wide tile count
    const int64_t g = g0 + gl;
    ProjState st;
    float4 cg = make_float4(0.f, 0.f, 0.f, 0.f);
    // opacity-only quantities, the same for every view: the radius scale
    // k = min(3, sqrt(2 ln(255 o))) and tau = 2 (ln(255 o) + margin)
    float k_sig = 0.f, tau = -1.f;
    if (valid) {
        project_base(P, stride, g, st);
        cg = make_float4(P[11 * stride + g], P[12 * stride + g], P[13 * stride + g], st.opac);
        if (st.opac >= kAlphaMin) {
            const float ln255o = logf(255.f * st.opac);
            k_sig = fminf(kRadiusSigmas, sqrtf(2.f * ln255o));
            tau = 2.f * (ln255o + kCullMargin);
        }
    }
    for (int v = v_begin; v < v_end; v++) {
        TileTest tt = {};
        bool has_tiles = false;
        int64_t item = 0;
        int4 rc = make_int4(0, 0, 0, 0);
        if (valid) {
            item = view_item_offset[v] - view_item_offset[vb] + gl;
            const vbm_camera cam = cams[v];
            project_view(cam, st);
            SplatRec sr;
            sr.c = cg;
            // A splat whose opacity is below the 1/255 compositing cut-off can never be
            // blended (alpha = o G <= o), so it gets no tiles.
            if (!st.culled && st.opac >= kAlphaMin) {
                float inv_det = 1.0f / st.det;
                float A = st.c * inv_det, B = -st.b * inv_det, C = st.a * inv_det;
                float mid = 0.5f * (st.a + st.c);
                float disc = mid * mid - st.det;
                float lam1 = mid + sqrtf(fmaxf(disc, kEigFloor));
                // Extent of the ellipse where o e^power >= 1/255 (capped at 3 sigma):
                // pixels beyond it skip this splat anyway, so fewer tiles list it.
                // Bounded so the integer rectangle arithmetic cannot overflow; any
                // radius above 2^24 already spans every image narrower than 6.7M px.
                float r = fminf(ceilf(k_sig * sqrtf(lam1)), 16777216.0f);
                float u = cam.fx * st.xz + cam.cx;
                float vv = cam.fy * st.yz + cam.cy;
                sr.g = make_float4(u, vv, A, B);
                // For the tile test and the compositing kernels' culling: tau =
                // 2 (ln(255 o) + margin); the bounding box of {q <= tau} has
                // half-widths sqrt(tau a) and sqrt(tau c) (the conic's determinant is
                // 1 / det), slightly widened; the edge minimisers' ratios B / C and
                // B / A are rounded divisions of the stored conic.
                const float bc = __fdiv_rn(B, C), ba = __fdiv_rn(B, A);
                sr.cu = make_float4(sqrtf(tau * st.a) * 1.0001f + 1e-3f, sqrtf(tau * st.c) * 1.0001f + 1e-3f, bc,
                                    ba);
                const int r_int = (int)r;
                sr.x = make_float4(C, tau, st.t[2], __int_as_float(r_int));
                int fu = (int)floorf(clampf(u, -kCoordClamp, kCoordClamp));
                int fv = (int)floorf(clampf(vv, -kCoordClamp, kCoordClamp));
                // floor division by the tile size, a power of two: arithmetic shifts
                const int lw = __ffs(tw) - 1, lh = __ffs(th) - 1;
                rc.x = min(max((fu - r_int) >> lw, 0), TX);
                rc.z = min(max(((fu + r_int) >> lw) + 1, 0), TX);
                rc.y = min(max((fv - r_int) >> lh, 0), TY);
                rc.w = min(max(((fv + r_int) >> lh) + 1, 0), TY);
                tt = TileTest{u, vv, A, B, C, bc, ba, tau, rc};
                has_tiles = true;
            } else {
                sr.g = make_float4(0.f, 0.f, 0.f, 0.f);
                sr.cu = make_float4(0.f, 0.f, 0.f, 0.f);
                sr.x = make_float4(0.f, -1.f, st.t[2], __int_as_float(0));
            }
            rec[item] = sr;
            if (gs) {   // the item's splat-gradient record, zero for the backward's atomics
                const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
                gs[3 * item] = z;
                gs[3 * item + 1] = z;
                gs[3 * item + 2] = z;
            }
        }
        // tiles of the rectangle that pass the exact tile test (the image size is
        // the plan's, as in the pair placement, so both take the same decisions),
        // counted per tile and recorded per item for the placement
        uint32_t n_listed = 0;
        const uint32_t word = listed_tiles(has_tiles, tt, tw, th, W, H, tile_count,
                                           (uint32_t)(v - vb) * (uint32_t)(TX * TY), TX, &n_listed);
        if (valid) {
            place[item] = pack_place(rc, word, st.t[2]);
            if (touched) touched[item] = n_listed;   // pairs of the item (radix-sort ordering)
        }
    }
}

// Adam step of one Gaussian's 14 parameters with gradient g14 (zero when
// !seen), in place in P, M, V ([14][stride]); non-finite gradient elements
// leave their scalars unchanged and are counted.  Rows go in two batches of
// seven, each batch's loads issued before its stores (the three arrays may
// alias as far as the compiler knows, so it would not move a later row's
// loads above an earlier row's stores).
__device__ __forceinline__ void adam_gaussian(const AdamArgs &a, int64_t stride, int64_t g, const float (&g14)[14],
                                              bool seen)
{
    const float2 bc = adam_bias_corrections(*a.step, a.beta1, a.beta2);
    uint32_t bad = 0;
#pragma unroll
    for (int k0 = 0; k0 < 14; k0 += 7) {
        float p[7], m[7], v[7];
#pragma unroll
        for (int k = 0; k < 7; k++) {
            const int64_t e = (k0 + k) * stride + g;
            p[k] = a.P[e];
            m[k] = a.M[e];
            v[k] = a.V[e];
        }
#pragma unroll
        for (int k = 0; k < 7; k++) {
            const bool ok = adam_elem(p[k], m[k], v[k], seen ? g14[k0 + k] : 0.f,
                                      adam_row_lr(k0 + k, a.lr[0], a.lr[1], a.lr[2], a.lr[3], a.lr[4]), a.beta1,
                                      a.beta2, a.eps, bc.x, bc.y);
            bad += !ok;
            if (!ok) continue;
            const int64_t e = (k0 + k) * stride + g;
            a.P[e] = p[k];
            a.M[e] = m[k];
            a.V[e] = v[k];
        }
    }
    if (bad && a.nonfinite) atomicAdd(a.nonfinite, bad);
}

// Chain rule from the per-item splat gradient (du, dv, dA, dB, dC, dopacity,
// dr, dg, db) to the 14 parameters, summed over the views of the call that
// see Gaussian g.  Mirrors the forward step by step (see the header comment).
// ADAM: the gradient is not written; the thread applies the Adam step to its
// Gaussian's parameters instead (Gaussians [0, a.n); those outside
// [g_begin, g_end) have a zero gradient), with the separate Adam kernel's
// arithmetic, so the result equals a backward with accumulate = 0 into a
// zeroed gradient followed by that kernel, bit for bit.
// Twenty resident one-warp blocks (at most 102 registers; the Adam epilogue
// would otherwise take 115 and leave 17): the kernel waits on its gradient
// loads.
template <bool ADAM>
__global__ void __launch_bounds__(32, 20) k_preprocess_bwd(const float *P, int64_t stride, const vbm_camera *__restrict__ cams,
                                 const int64_t *__restrict__ scene_offset, int n_scenes,
                                 const int32_t *__restrict__ scene_view_ptr, const int32_t *__restrict__ scene_views,
                                 const int64_t *__restrict__ view_item_offset, int vb, int vc,
                                 const float *__restrict__ gs, float *__restrict__ grad, int accumulate,
                                 int64_t g_begin, int64_t g_end, AdamArgs a)
{
    const int64_t g = (ADAM ? 0 : g_begin) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ADAM ? g >= a.n : g >= g_end) return;
    if (ADAM && (g < g_begin || g >= g_end)) {   // no view of the call renders g's scene
        const float zero[14] = {};
        adam_gaussian(a, stride, g, zero, false);
        return;
    }
    int lo = 0, hi = n_scenes - 1;  // scene of g: last s with scene_offset[s] <= g
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (scene_offset[mid] <= g) lo = mid; else hi = mid - 1;
    }
    const int scene = lo;
    const int64_t gl = g - scene_offset[scene];
    float acc[14];
#pragma unroll
    for (int k = 0; k < 14; k++) acc[k] = 0.f;
    // dL/dSigma + its transpose, summed over the views: the scale and rotation
    // gradients are linear in it, so they are formed once after the loop
    float GS2[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) GS2[i][j] = 0.f;
    ProjState st;
    project_base(P, stride, g, st);
    bool seen = false;
    for (int e = scene_view_ptr[scene]; e < scene_view_ptr[scene + 1]; e++) {
        const int v = scene_views[e];
        if (v < vb || v >= vb + vc) continue;
        seen = true;
        const int64_t item = view_item_offset[v] - view_item_offset[vb] + gl;
        float g9[9];
#pragma unroll
        for (int k = 0; k < 9; k++) g9[k] = gs[item * kGradStride + k];
        const vbm_camera cam = cams[v];
        project_view(cam, st);
        acc[10] += g9[5] * st.opac * (1.f - st.opac);
        acc[11] += g9[6];
        acc[12] += g9[7];
        acc[13] += g9[8];
        if (st.culled) continue;
        const float *Wm = cam.R;
        float a = st.a, b = st.b, c = st.c, D = st.det;
        float iD2 = 1.0f / (D * D);
        float dA = g9[2], dB = g9[3], dC = g9[4];
        float dLa = (dA * (-c * c) + dB * (b * c) + dC * (-b * b)) * iD2;
        float dLb = (dA * (2.f * b * c) + dB * (-(a * c + b * b)) + dC * (2.f * a * b)) * iD2;
        float dLc = (dA * (-b * b) + dB * (a * b) + dC * (-a * a)) * iD2;
        float ST0[3], ST1[3];
#pragma unroll
        for (int i = 0; i < 3; i++) {
            ST0[i] = st.Sig[i][0] * st.T0[0] + st.Sig[i][1] * st.T0[1] + st.Sig[i][2] * st.T0[2];
            ST1[i] = st.Sig[i][0] * st.T1[0] + st.Sig[i][1] * st.T1[1] + st.Sig[i][2] * st.T1[2];
        }
        float dT0[3], dT1[3];
#pragma unroll
        for (int i = 0; i < 3; i++) {
            dT0[i] = 2.f * dLa * ST0[i] + dLb * ST1[i];
            dT1[i] = dLb * ST0[i] + 2.f * dLc * ST1[i];
        }
        float dJ00 = dT0[0] * Wm[0] + dT0[1] * Wm[1] + dT0[2] * Wm[2];
        float dJ02 = dT0[0] * Wm[6] + dT0[1] * Wm[7] + dT0[2] * Wm[8];
        float dJ11 = dT1[0] * Wm[3] + dT1[1] * Wm[4] + dT1[2] * Wm[5];
        float dJ12 = dT1[0] * Wm[6] + dT1[1] * Wm[7] + dT1[2] * Wm[8];
        float tx = st.t[0], ty = st.t[1];
        float itz = st.itz, itz2 = itz * itz;
        float dxc_dtx = st.clampx ? 0.f : itz, dxc_dtz = st.clampx ? 0.f : -tx * itz2;
        float dyc_dty = st.clampy ? 0.f : itz, dyc_dtz = st.clampy ? 0.f : -ty * itz2;
        float fx = cam.fx, fy = cam.fy;
        float dt0 = g9[0] * fx * itz + dJ02 * (-fx * itz) * dxc_dtx;
        float dt1 = g9[1] * fy * itz + dJ12 * (-fy * itz) * dyc_dty;
        float dt2 = g9[0] * (-fx * tx * itz2) + g9[1] * (-fy * ty * itz2) + dJ00 * (-fx * itz2) +
                    dJ11 * (-fy * itz2) + dJ02 * (fx * st.xzc * itz2 - fx * itz * dxc_dtz) +
                    dJ12 * (fy * st.yzc * itz2 - fy * itz * dyc_dtz);
#pragma unroll
        for (int k = 0; k < 3; k++) acc[k] += Wm[k] * dt0 + Wm[3 + k] * dt1 + Wm[6 + k] * dt2;
        // dL/dSigma = dLa T0 T0^T + dLb T0 T1^T + dLc T1 T1^T; add it and its transpose
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++)
                GS2[i][j] += 2.f * dLa * st.T0[i] * st.T0[j] + dLb * (st.T0[i] * st.T1[j] + st.T1[i] * st.T0[j]) +
                             2.f * dLc * st.T1[i] * st.T1[j];
    }
    if (seen) {
        // Sigma = M M^T with M = R diag(s): dL/dM = (G + G^T) M
        float dR[3][3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            float ds = 0.f;
#pragma unroll
            for (int i = 0; i < 3; i++) {
                float dM = 0.f;
#pragma unroll
                for (int j = 0; j < 3; j++) dM += GS2[i][j] * st.R[j][k] * st.s[k];
                ds += dM * st.R[i][k];
                dR[i][k] = dM * st.s[k];
            }
            acc[3 + k] += ds * st.s[k];
        }
        float w = st.qn[0], x = st.qn[1], y = st.qn[2], z = st.qn[3];
        float dq[4];
        dq[0] = 2.f * (-z * dR[0][1] + y * dR[0][2] + z * dR[1][0] - x * dR[1][2] - y * dR[2][0] + x * dR[2][1]);
        dq[1] = 2.f * (y * dR[0][1] + z * dR[0][2] + y * dR[1][0] - 2.f * x * dR[1][1] - w * dR[1][2] +
                       z * dR[2][0] + w * dR[2][1] - 2.f * x * dR[2][2]);
        dq[2] = 2.f * (-2.f * y * dR[0][0] + x * dR[0][1] + w * dR[0][2] + x * dR[1][0] + z * dR[1][2] -
                       w * dR[2][0] + z * dR[2][1] - 2.f * y * dR[2][2]);
        dq[3] = 2.f * (-2.f * z * dR[0][0] - w * dR[0][1] + x * dR[0][2] + w * dR[1][0] - 2.f * z * dR[1][1] +
                       y * dR[1][2] + x * dR[2][0] + y * dR[2][1]);
        float dot = dq[0] * st.qn[0] + dq[1] * st.qn[1] + dq[2] * st.qn[2] + dq[3] * st.qn[3];
        float iq = 1.0f / st.qnorm;
#pragma unroll
        for (int k = 0; k < 4; k++) acc[6 + k] += (dq[k] - st.qn[k] * dot) * iq;
    }
    if constexpr (ADAM) {
        adam_gaussian(a, stride, g, acc, seen);
        return;
    }
    if (!seen) return;
#pragma unroll
    for (int k = 0; k < 14; k++) {
        float *dst = grad + k * stride + g;
        *dst = accumulate ? *dst + acc[k] : acc[k];
    }
}

}  // namespace

vbm_status preprocess_fwd(vbm_plan *p, const float *params, int64_t stride, const vbm_camera *cams, int vb, int vc,
                          cudaStream_t st)
{
    if (p->max_scene == 0) return VBM_OK;
    // views per thread: as many as keep about four waves of threads (the
    // view-independent state is then built once per Gaussian and view group)
    int vpt = 1;
    if (p->desc.n_scenes == 1) {
        const int64_t wave = (int64_t)num_sms() * 2048;
        vpt = (int)std::max<int64_t>(1, std::min<int64_t>(vc, p->max_scene * vc / (4 * wave)));
    }
    dim3 block(256);
    dim3 grid((unsigned)((p->max_scene + 255) / 256), (unsigned)((vc + vpt - 1) / vpt));
    // plans that have run a backward get their splat-gradient records zeroed
    // here (render-only plans skip the writes; a plan's first backward clears
    // them itself)
    float4 *gs = p->bwd_seen ? reinterpret_cast<float4 *>(p->g_splat) : nullptr;
    auto kernel = vpt > 1 ? k_preprocess_fwd<true> : k_preprocess_fwd<false>;
    kernel<<<grid, block, 0, st>>>(params, stride, cams, p->d_scene_offset,
                                   p->desc.n_scenes > 1 ? p->d_view_scene : nullptr, p->d_view_item_offset, vb, vc,
                                   vpt, p->TX, p->TY, p->desc.tile_w, p->desc.tile_h, p->desc.width, p->desc.height,
                                   p->rec, gs, p->place, p->tile_count, p->touched);
    VBM_LAUNCH("preprocess_fwd");
    note_launches(1);
    return VBM_OK;
}

vbm_status preprocess_bwd(vbm_plan *p, const float *params, int64_t stride, const vbm_camera *cams, int vb, int vc,
                          float *grad, int accumulate, cudaStream_t st, const AdamArgs *adam)
{
    // Gaussians of the scenes the call's views render form one column range
    // when the views are consecutive; bound it by the scenes' extent.
    int64_t g_begin = INT64_MAX, g_end = 0;
    for (int v = vb; v < vb + vc; v++) {
        int s = p->desc.n_scenes > 1 ? p->view_scene[v] : 0;
        g_begin = std::min(g_begin, p->scene_offset[s]);
        g_end = std::max(g_end, p->scene_offset[s + 1]);
    }
    if (g_end <= g_begin && !adam) return VBM_OK;
    int64_t n = g_end - g_begin;
    // one-warp blocks: a thread's work (its Gaussian's views) is long and the
    // blocks are few, so the finest granularity keeps the SMs evenly loaded
    // (with 128-thread blocks the 8 x 512^2 workload left a second wave of 19
    // blocks running on 19 SMs)
    if (adam) {   // every Gaussian of [0, n) takes its Adam step
        const int64_t na = adam->n;
        if (na == 0) return VBM_OK;
        k_preprocess_bwd<true><<<(unsigned)((na + 31) / 32), 32, 0, st>>>(
            params, stride, cams, p->d_scene_offset, p->desc.n_scenes, p->d_scene_view_ptr, p->d_scene_views,
            p->d_view_item_offset, vb, vc, p->g_splat, nullptr, 0, g_begin, std::min(g_end, na), *adam);
    } else {
        k_preprocess_bwd<false><<<(unsigned)((n + 31) / 32), 32, 0, st>>>(
            params, stride, cams, p->d_scene_offset, p->desc.n_scenes, p->d_scene_view_ptr, p->d_scene_views,
            p->d_view_item_offset, vb, vc, p->g_splat, grad, accumulate, g_begin, g_end, AdamArgs{});
    }
    VBM_LAUNCH("preprocess_bwd");
    note_launches(1);
    return VBM_OK;
}

}  // namespace vbm
