// Volume -> Gaussians (Sec. 4.1-4.3): transfer function, periodised 3D DWT,
// adaptive coefficient filtering (Supp. Sec. 1) and the per-coefficient map
// (Eq. 22-24).  A setup step, run once per volume and TF.
//
// DWT: one level = three axis passes (x, y, z), each a gather kernel with one
// thread per output coefficient (9- and 7-tap filters from constant memory;
// neighbouring threads read neighbouring inputs, so the taps hit L1/L2).
//
// Selection per subband, all on the device except the budget allocation
// (one copy of the 7J+1 subband energies to the host):
//   v = sqrt(((a0 a0 + a1 a1) + a2 a2) + a3 a3) in IEEE float32, rounded op by
//   op (explicit __fmul_rn/__fadd_rn/__fsqrt_rn, so the order is fixed);
//   medians and the K-th largest value by radix select on the float bits (v >= 0
//   so the bits order like the values): four 8-bit histogram passes, no sort;
//   sigma = MAD / 0.6745 and T = lambda sigma in float32;
//   keep = v >= max(T, v_(K')) and v > 0.
// Kept coefficients are compacted in raster order of each subband by a
// block scan and mapped to the P[14][capacity] layout.
#include <cmath>
#include <map>
#include <vector>

#include "vbm_internal.h"

namespace vbm {

namespace {

struct DevFilters {
    int lo_n0, lo_len, hi_n0, hi_len;
    float lo[16], hi[16];
};
__constant__ DevFilters c_filt;

struct TFDev {
    int n;
    float x[16];
    float rgba[16][4];
};

__global__ void k_tf_apply(const float *__restrict__ F, int64_t n, TFDev tf, float *__restrict__ RF)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float f = fminf(fmaxf(F[i], 0.f), 1.f);
        float out[4];
        if (f <= tf.x[0]) {
            for (int c = 0; c < 4; c++) out[c] = tf.rgba[0][c];
        } else if (f >= tf.x[tf.n - 1]) {
            for (int c = 0; c < 4; c++) out[c] = tf.rgba[tf.n - 1][c];
        } else {
            int k = 0;
            while (k < tf.n - 2 && tf.x[k + 1] <= f) k++;
            const float t = (f - tf.x[k]) / (tf.x[k + 1] - tf.x[k]);
            for (int c = 0; c < 4; c++) out[c] = (1.f - t) * tf.rgba[k][c] + t * tf.rgba[k + 1][c];
        }
        for (int c = 0; c < 4; c++) RF[c * n + i] = out[c];
    }
}

// One periodised analysis pass along `axis` over the region [0,s0)x[0,s1)x[0,s2)
// of arrays with row strides (nx, nx*ny): output index k < L/2 is the
// low-pass a[k], k >= L/2 the high-pass d[k - L/2].
__global__ void k_dwt_axis(const float *__restrict__ src, float *__restrict__ dst, int nx, int ny, int sx, int sy,
                           int sz, int axis)
{
    const int64_t total = (int64_t)sx * sy * sz;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % sx);
        const int y = (int)((i / sx) % sy);
        const int z = (int)(i / ((int64_t)sx * sy));
        int c[3] = {x, y, z};
        const int L = axis == 0 ? sx : axis == 1 ? sy : sz;
        const int half = L >> 1;
        const int k = c[axis];
        const bool low = k < half;
        const int kk = low ? k : k - half;
        const int n0 = low ? c_filt.lo_n0 : c_filt.hi_n0;
        const int len = low ? c_filt.lo_len : c_filt.hi_len;
        const int base = 2 * kk + (low ? 0 : 1);
        float acc = 0.f;
        for (int t = 0; t < len; t++) {
            int m = base + n0 + t;
            m %= L;
            if (m < 0) m += L;
            c[axis] = m;
            const float w = low ? c_filt.lo[t] : c_filt.hi[t];
            acc += w * src[((int64_t)c[2] * ny + c[1]) * nx + c[0]];
        }
        dst[((int64_t)z * ny + y) * nx + x] = acc;
    }
}

// ----------------------------------------------------------------- select

struct SubStat {
    float med, mad, T, thr;
    float sel_a, sel_b;          // scratch of the two order statistics of a median
    int64_t count_c;             // |C|
    int64_t k;                   // rank of the running selection
    uint32_t prefix, mask;
    int64_t kept;
};

__global__ void k_energy(const float *__restrict__ A, int nx, int ny, int ox, int oy, int oz, int mx, int my, int mz,
                         double *__restrict__ E)
{
    __shared__ double red[256];
    const int64_t total = (int64_t)mx * my * mz;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % mx), y = (int)((i / mx) % my), z = (int)(i / ((int64_t)mx * my));
        const double a = A[((int64_t)(oz + z) * ny + (oy + y)) * nx + (ox + x)];
        s += a * a;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < (unsigned)off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(E, red[0]);
}

__global__ void k_joint_mag(const float *__restrict__ A, int64_t chan, int nx, int ny, int ox, int oy, int oz, int mx,
                            int my, int mz, float *__restrict__ v)
{
    const int64_t total = (int64_t)mx * my * mz;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % mx), y = (int)((i / mx) % my), z = (int)(i / ((int64_t)mx * my));
        const int64_t e = ((int64_t)(oz + z) * ny + (oy + y)) * nx + (ox + x);
        const float a0 = A[e], a1 = A[chan + e], a2 = A[2 * chan + e], a3 = A[3 * chan + e];
        float acc = __fmul_rn(a0, a0);
        acc = __fadd_rn(acc, __fmul_rn(a1, a1));
        acc = __fadd_rn(acc, __fmul_rn(a2, a2));
        acc = __fadd_rn(acc, __fmul_rn(a3, a3));
        v[i] = __fsqrt_rn(acc);
    }
}

__global__ void k_abs_dev(const float *__restrict__ v, int64_t n, const SubStat *__restrict__ st,
                          float *__restrict__ dev)
{
    const float med = st->med;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dev[i] = fabsf(__fsub_rn(v[i], med));
}

// radix select: histogram of the digit at `shift` among elements matching the prefix
__global__ void k_sel_hist(const float *__restrict__ v, int64_t n, const SubStat *__restrict__ st, int shift,
                           uint32_t *__restrict__ hist)
{
    __shared__ uint32_t h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const uint32_t prefix = st->prefix, mask = st->mask;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t b = __float_as_uint(v[i]);
        if ((b & mask) == prefix) atomicAdd(&h[(b >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

__global__ void k_sel_pick(SubStat *st, const uint32_t *__restrict__ hist, int shift)
{
    if (threadIdx.x || blockIdx.x) return;
    int64_t k = st->k;
    uint32_t d = 0;
    for (; d < 256; d++) {
        if (k < (int64_t)hist[d]) break;
        k -= hist[d];
    }
    st->k = k;
    st->prefix |= d << shift;
    st->mask |= 255u << shift;
}

// which: 0 = k fixed (host), 1 = k = n - K' (K-th largest among candidates)
__global__ void k_sel_begin(SubStat *st, int64_t k, int which, int64_t n, int64_t K)
{
    if (threadIdx.x || blockIdx.x) return;
    if (which == 1) {
        const int64_t Kp = min(K, st->count_c);
        k = Kp > 0 ? n - Kp : 0;
    }
    st->k = k;
    st->prefix = 0;
    st->mask = 0;
}

// where: 0 -> sel_a, 1 -> sel_b
__global__ void k_sel_store(SubStat *st, int where)
{
    if (threadIdx.x || blockIdx.x) return;
    const float val = __uint_as_float(st->prefix);
    if (where == 0) st->sel_a = val; else st->sel_b = val;
}

// role: 0 = median of v -> med, 1 = median of dev -> mad (then sigma, T)
__global__ void k_median_done(SubStat *st, int even, int role, float lambda)
{
    if (threadIdx.x || blockIdx.x) return;
    const float m = even ? __fmul_rn(__fadd_rn(st->sel_a, st->sel_b), 0.5f) : st->sel_b;
    if (role == 0) {
        st->med = m;
    } else {
        st->mad = m;
        const float sigma = __fdiv_rn(m, 0.6745f);
        st->T = __fmul_rn(lambda, sigma);
    }
}

__global__ void k_count_ge(const float *__restrict__ v, int64_t n, SubStat *st)
{
    __shared__ unsigned long long red;
    if (threadIdx.x == 0) red = 0;
    __syncthreads();
    const float T = st->T;
    unsigned long long c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += v[i] >= T;
    atomicAdd(&red, c);
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd((unsigned long long *)&st->count_c, red);
}

__global__ void k_threshold(SubStat *st, int64_t K)
{
    if (threadIdx.x || blockIdx.x) return;
    const int64_t Kp = min(K, st->count_c);
    st->thr = Kp > 0 ? fmaxf(st->T, __uint_as_float(st->prefix)) : __int_as_float(0x7f800000);
}

__global__ void k_flags(const float *__restrict__ v, int nx, int ny, int ox, int oy, int oz, int mx, int my, int mz,
                        SubStat *st, uint8_t *__restrict__ keep)
{
    __shared__ unsigned long long red;
    if (threadIdx.x == 0) red = 0;
    __syncthreads();
    const float thr = st->thr;
    const int64_t total = (int64_t)mx * my * mz;
    unsigned long long c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % mx), y = (int)((i / mx) % my), z = (int)(i / ((int64_t)mx * my));
        const bool k = v[i] >= thr && v[i] > 0.f;
        keep[((int64_t)(oz + z) * ny + (oy + y)) * nx + (ox + x)] = k;
        c += k;
    }
    atomicAdd(&red, c);
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd((unsigned long long *)&st->kept, red);
}

// ------------------------------------------------------------------ map

struct MapEntry {
    float u[3];
    float w;
    float log_scale[3];
    float quat[4];
    float s;        // 2^{-3j/2} or 1
    int j;
};

// Single-block ordered compaction of one subband (raster order), then the
// per-coefficient map of Eq. 22-24.  One block per subband keeps the order
// without a global scan; blocks walk their subband in chunks of blockDim.
__global__ void __launch_bounds__(1024) k_map_subband(const float *__restrict__ A, int64_t chan, int nx, int ny,
                                                      int ox, int oy, int oz, int mx, int my, int mz,
                                                      const uint8_t *__restrict__ keep, MapEntry me, int64_t out_off,
                                                      float *__restrict__ P, int64_t stride)
{
    __shared__ int warp_tot[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int64_t total = (int64_t)mx * my * mz;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int64_t base = 0; base < total; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        int x = 0, y = 0, z = 0;
        bool k = false;
        int64_t e = 0;
        if (i < total) {
            x = (int)(i % mx); y = (int)((i / mx) % my); z = (int)(i / ((int64_t)mx * my));
            e = ((int64_t)(oz + z) * ny + (oy + y)) * nx + (ox + x);
            k = keep[e] != 0;
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, k);
        if (lane == 0) warp_tot[warp] = __popc(bal);
        __syncthreads();
        int before = 0, all = 0;
        for (int w = 0; w < nwarps; w++) {
            if (w < warp) before += warp_tot[w];
            all += warp_tot[w];
        }
        if (k) {
            const int64_t pos = out_off + carry + before + __popc(bal & ((1u << lane) - 1u));
            float amp[4];
            for (int c = 0; c < 4; c++) amp[c] = me.s * fabsf(A[c * chan + e]) * me.w;
            const float step = (float)(1 << me.j);
            P[0 * stride + pos] = me.u[0] + step * x + 0.5f;
            P[1 * stride + pos] = me.u[1] + step * y + 0.5f;
            P[2 * stride + pos] = me.u[2] + step * z + 0.5f;
            for (int d = 0; d < 3; d++) P[(3 + d) * stride + pos] = me.log_scale[d];
            for (int d = 0; d < 4; d++) P[(6 + d) * stride + pos] = me.quat[d];
            // floor 2/255: a retained coefficient stays above the 1/255 cut-off
            const float op = fminf(fmaxf(amp[3], 2.f / 255.f), 0.99f);
            P[10 * stride + pos] = logf(op / (1.f - op));
            P[11 * stride + pos] = amp[0];
            P[12 * stride + pos] = amp[1];
            P[13 * stride + pos] = amp[2];
        }
        __syncthreads();
        if (threadIdx.x == 0) carry += all;
        __syncthreads();
    }
}

// ------------------------------------------------------------- helpers

vbm_status upload_filters(int wavelet)
{
    FilterBank fb = make_filters(wavelet);
    DevFilters f{};
    f.lo_n0 = fb.ht.begin()->first;
    f.lo_len = (int)fb.ht.size();
    f.hi_n0 = fb.gt.begin()->first;
    f.hi_len = (int)fb.gt.size();
    int t = 0;
    for (auto &kv : fb.ht) f.lo[t++] = (float)kv.second;
    t = 0;
    for (auto &kv : fb.gt) f.hi[t++] = (float)kv.second;
    VBM_CUDA(cudaMemcpyToSymbol(c_filt, &f, sizeof(f)));
    return VBM_OK;
}

TFDev to_dev(const vbm_tf *tf)
{
    TFDev t{};
    t.n = tf->n_knots;
    for (int i = 0; i < 16; i++) {
        t.x[i] = tf->x[i];
        for (int c = 0; c < 4; c++) t.rgba[i][c] = tf->rgba[i][c];
    }
    return t;
}

int grid_for(int64_t n, int threads = 256)
{
    int64_t b = (n + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms() * 16;
    return (int)std::max<int64_t>(1, std::min(b, cap));
}

vbm_status dwt_channels(float *data, int n_channels, const int dims[3], int levels, int wavelet, float *tmp,
                        cudaStream_t st)
{
    vbm_status s = upload_filters(wavelet);
    if (s != VBM_OK) return s;
    const int nx = dims[0], ny = dims[1], nz = dims[2];
    const int64_t n = (int64_t)nx * ny * nz;
    float *t1 = tmp, *t2 = tmp + n;
    for (int c = 0; c < n_channels; c++) {
        float *P = data + c * n;
        for (int j = 1; j <= levels; j++) {
            const int sx = nx >> (j - 1), sy = ny >> (j - 1), sz = nz >> (j - 1);
            const int64_t tot = (int64_t)sx * sy * sz;
            const int g = grid_for(tot);
            k_dwt_axis<<<g, 256, 0, st>>>(P, t1, nx, ny, sx, sy, sz, 0);
            k_dwt_axis<<<g, 256, 0, st>>>(t1, t2, nx, ny, sx, sy, sz, 1);
            k_dwt_axis<<<g, 256, 0, st>>>(t2, P, nx, ny, sx, sy, sz, 2);
            VBM_LAUNCH("dwt_axis");
        }
    }
    return VBM_OK;
}

struct Band {
    int j, o[3], ox, oy, oz, mx, my, mz;
    int64_t n;
};

std::vector<Band> bands_of(const int dims[3], int levels)
{
    std::vector<Band> out;
    for (int j = 1; j <= levels; j++)
        for (int code = 0; code < 8; code++) {
            if (code == 0 && j != levels) continue;
            Band b;
            b.j = j;
            b.o[0] = code & 1; b.o[1] = (code >> 1) & 1; b.o[2] = (code >> 2) & 1;
            b.mx = dims[0] >> j; b.my = dims[1] >> j; b.mz = dims[2] >> j;
            b.ox = b.o[0] * b.mx; b.oy = b.o[1] * b.my; b.oz = b.o[2] * b.mz;
            b.n = (int64_t)b.mx * b.my * b.mz;
            out.push_back(b);
        }
    return out;
}

// k-th smallest (0-based, k set by k_sel_begin) of v[0..n) into st->prefix
void radix_select(const float *v, int64_t n, SubStat *st, uint32_t *hist, cudaStream_t s)
{
    const int g = grid_for(n);
    for (int shift = 24; shift >= 0; shift -= 8) {
        cudaMemsetAsync(hist, 0, 256 * sizeof(uint32_t), s);
        k_sel_hist<<<g, 256, 0, s>>>(v, n, st, shift, hist);
        k_sel_pick<<<1, 32, 0, s>>>(st, hist, shift);
    }
}

void median_of(const float *v, int64_t n, SubStat *st, uint32_t *hist, int role, float lambda, cudaStream_t s)
{
    const bool even = (n % 2) == 0;
    if (even) {
        k_sel_begin<<<1, 32, 0, s>>>(st, n / 2 - 1, 0, n, 0);
        radix_select(v, n, st, hist, s);
        k_sel_store<<<1, 32, 0, s>>>(st, 0);
    }
    k_sel_begin<<<1, 32, 0, s>>>(st, n / 2, 0, n, 0);
    radix_select(v, n, st, hist, s);
    k_sel_store<<<1, 32, 0, s>>>(st, 1);
    k_median_done<<<1, 32, 0, s>>>(st, even ? 1 : 0, role, lambda);
}

}  // namespace

size_t build_workspace_bytes(const int dims[3], int levels)
{
    const size_t n = (size_t)dims[0] * dims[1] * dims[2];
    size_t b = 0;
    auto add = [&](size_t bytes) { b += (bytes + 255) / 256 * 256; };
    add(4 * n * sizeof(float));         // RF / pyramid
    add(2 * n * sizeof(float));         // DWT temporaries (reused as v, dev)
    add(n);                             // keep flags
    add(64 * sizeof(SubStat));
    add(64 * sizeof(double));
    add(256 * sizeof(uint32_t));
    (void)levels;
    return b;
}

}  // namespace vbm

using namespace vbm;

extern "C" {

vbm_status vbm_tf_apply(const float *d_volume, int64_t n, const vbm_tf *tf, float *d_rf, void *stream)
{
    VBM_ARG(d_volume && tf && d_rf && n >= 0, "invalid argument");
    VBM_ARG(tf->n_knots >= 2 && tf->n_knots <= 16, "n_knots must be in [2, 16]");
    for (int i = 1; i < tf->n_knots; i++) VBM_ARG(tf->x[i] > tf->x[i - 1], "TF knots must be ascending");
    if (n == 0) return VBM_OK;
    k_tf_apply<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(d_volume, n, to_dev(tf), d_rf);
    VBM_LAUNCH("tf_apply");
    return VBM_OK;
}

vbm_status vbm_dwt3d(float *d_data, int n_channels, const int dims[3], int levels, int wavelet, float *d_tmp,
                     void *stream)
{
    VBM_ARG(d_data && dims && d_tmp && n_channels >= 1, "invalid argument");
    VBM_ARG(levels >= 1 && levels <= 9, "levels must be in [1, 9]");
    VBM_ARG(wavelet == 0 || wavelet == 1, "wavelet must be 0 or 1");
    for (int d = 0; d < 3; d++)
        VBM_ARG(dims[d] > 0 && dims[d] % (1 << levels) == 0, "dims must be divisible by 2^levels");
    return dwt_channels(d_data, n_channels, dims, levels, wavelet, d_tmp, (cudaStream_t)stream);
}

vbm_status vbm_build_workspace_size(const int dims[3], int levels, size_t *bytes)
{
    VBM_ARG(dims && bytes, "null argument");
    *bytes = build_workspace_bytes(dims, levels);
    return VBM_OK;
}

vbm_status vbm_build(const float *d_volume, const int dims[3], const vbm_tf *tf, const vbm_bank *bank,
                     const vbm_select *sel, float *d_params, int64_t capacity, int64_t *n_out, float *d_coef,
                     uint8_t *d_keep, void *d_ws, size_t ws_bytes, void *stream)
{
    VBM_ARG(d_volume && dims && tf && bank && sel && n_out && d_ws, "null argument");
    VBM_ARG(capacity >= 0 && (capacity == 0 || d_params), "invalid params buffer");
    const int levels = bank->levels;
    VBM_ARG(levels >= 1 && levels <= 9 && bank->n_sub == 7 * levels + 1, "invalid bank");
    for (int d = 0; d < 3; d++)
        VBM_ARG(dims[d] > 0 && dims[d] % (1 << levels) == 0, "dims must be divisible by 2^levels");
    VBM_ARG(ws_bytes >= build_workspace_bytes(dims, levels), "build workspace too small");
    VBM_ARG(sel->K_tot > 0 && sel->min_per_band >= 0, "invalid selection parameters");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = (int64_t)dims[0] * dims[1] * dims[2];
    char *w = (char *)d_ws;
    auto take = [&](size_t bytes) {
        char *p = w;
        w += (bytes + 255) / 256 * 256;
        return (void *)p;
    };
    float *A = (float *)take(4 * n * sizeof(float));
    float *tmp = (float *)take(2 * n * sizeof(float));
    uint8_t *keep = (uint8_t *)take(n);
    SubStat *stats = (SubStat *)take(64 * sizeof(SubStat));
    double *E = (double *)take(64 * sizeof(double));
    uint32_t *hist = (uint32_t *)take(256 * sizeof(uint32_t));

    vbm_status s = vbm_tf_apply(d_volume, n, tf, A, stream);
    if (s != VBM_OK) return s;
    s = dwt_channels(A, 4, dims, levels, bank->wavelet, tmp, st);
    if (s != VBM_OK) return s;
    std::vector<Band> bands = bands_of(dims, levels);
    const int nb = (int)bands.size();
    VBM_CUDA(cudaMemsetAsync(E, 0, 64 * sizeof(double), st));
    VBM_CUDA(cudaMemsetAsync(stats, 0, 64 * sizeof(SubStat), st));
    VBM_CUDA(cudaMemsetAsync(keep, 0, n, st));
    const float *alpha = A + 3 * n;
    for (int b = 0; b < nb; b++) {
        const Band &B = bands[b];
        k_energy<<<grid_for(B.n), 256, 0, st>>>(alpha, dims[0], dims[1], B.ox, B.oy, B.oz, B.mx, B.my, B.mz, E + b);
    }
    VBM_LAUNCH("energy");
    std::vector<double> hE(nb);
    VBM_CUDA(cudaMemcpyAsync(hE.data(), E, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    VBM_CUDA(cudaStreamSynchronize(st));
    // budget allocation (Supp. Sec. 1.1), host FP64
    std::vector<double> S(nb);
    double sumS = 0.0;
    for (int b = 0; b < nb; b++) {
        S[b] = std::pow(hE[b], sel->alpha_E) * std::pow((double)bands[b].n, sel->beta_N);
        sumS += S[b];
    }
    std::vector<int64_t> K(nb);
    for (int b = 0; b < nb; b++) {
        double share = sumS > 0 ? (double)sel->K_tot * S[b] / sumS : 0.0;
        K[b] = std::max<int64_t>(sel->min_per_band, (int64_t)std::floor(share));
    }
    float *v = tmp, *dev = tmp + n;
    const float lam = (float)sel->lambda_mad;
    for (int b = 0; b < nb; b++) {
        const Band &B = bands[b];
        SubStat *stb = stats + b;
        const int g = grid_for(B.n);
        k_joint_mag<<<g, 256, 0, st>>>(A, n, dims[0], dims[1], B.ox, B.oy, B.oz, B.mx, B.my, B.mz, v);
        median_of(v, B.n, stb, hist, 0, lam, st);
        k_abs_dev<<<g, 256, 0, st>>>(v, B.n, stb, dev);
        median_of(dev, B.n, stb, hist, 1, lam, st);
        k_count_ge<<<g, 256, 0, st>>>(v, B.n, stb);
        k_sel_begin<<<1, 32, 0, st>>>(stb, 0, 1, B.n, K[b]);
        radix_select(v, B.n, stb, hist, st);
        k_threshold<<<1, 32, 0, st>>>(stb, K[b]);
        k_flags<<<g, 256, 0, st>>>(v, dims[0], dims[1], B.ox, B.oy, B.oz, B.mx, B.my, B.mz, stb, keep);
        VBM_LAUNCH("select");
    }
    std::vector<SubStat> hs(nb);
    VBM_CUDA(cudaMemcpyAsync(hs.data(), stats, nb * sizeof(SubStat), cudaMemcpyDeviceToHost, st));
    VBM_CUDA(cudaStreamSynchronize(st));
    int64_t total = 0;
    std::vector<int64_t> off(nb);
    for (int b = 0; b < nb; b++) {
        off[b] = total;
        total += hs[b].kept;
    }
    *n_out = total;
    if (d_coef) VBM_CUDA(cudaMemcpyAsync(d_coef, A, 4 * n * sizeof(float), cudaMemcpyDeviceToDevice, st));
    if (d_keep) VBM_CUDA(cudaMemcpyAsync(d_keep, keep, n, cudaMemcpyDeviceToDevice, st));
    if (total > capacity) {
        VBM_CUDA(cudaStreamSynchronize(st));
        set_error("vbm_build: " + std::to_string(total) + " Gaussians kept, capacity " + std::to_string(capacity));
        return VBM_ERR_CAPACITY;
    }
    for (int b = 0; b < nb; b++) {
        const Band &B = bands[b];
        const vbm_bank_entry &e = bank->sub[b];
        VBM_ARG(e.j == B.j && e.o[0] == B.o[0] && e.o[1] == B.o[1] && e.o[2] == B.o[2], "bank order mismatch");
        MapEntry me;
        for (int d = 0; d < 3; d++) {
            me.u[d] = (float)e.u[d];
            me.log_scale[d] = e.log_scale[d];
        }
        for (int d = 0; d < 4; d++) me.quat[d] = e.quat[d];
        me.w = (float)e.w;
        me.j = B.j;
        me.s = sel->energy_comp ? (float)std::pow(2.0, -1.5 * B.j) : 1.f;
        if (hs[b].kept == 0) continue;
        k_map_subband<<<1, 1024, 0, st>>>(A, n, dims[0], dims[1], B.ox, B.oy, B.oz, B.mx, B.my, B.mz, keep, me,
                                          off[b], d_params, capacity);
        VBM_LAUNCH("map_subband");
    }
    VBM_CUDA(cudaStreamSynchronize(st));
    return VBM_OK;
}

}  // extern "C"
