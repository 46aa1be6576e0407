// Wavelet filters and the wavelet-to-Gaussian transition bank, host FP64.
//
// Filters.  bior4.4 is the Cohen-Daubechies-Feauveau pair with four
// vanishing moments per side: with x = sin^2(w/2) the low-pass product is
// cos^8(w/2) P(x), P(x) = 1 + 4x + 10x^2 + 20x^3; the 7-tap low-pass takes
// cos^4 and the linear factor of P's real root, the 9-tap low-pass cos^4 and
// the quadratic factor of its complex pair; both are scaled to sum sqrt(2).
// High-pass filters are the (-1)^n modulated low-pass filters of the other
// side.  Haar is given directly.
//
// Bank (Sec. 4.2).  The canonical kernel of subband (j, o) is the IDWT of a
// unit impulse in that subband (Eq. 9-10).  The 3D transform is separable, so
// that response is the outer product of three 1D level-j responses (the
// low-pass chain for o_d = L, the detail chain for o_d = H), each obtained by
// j periodised 1D synthesis steps on a grid of 2^j * 16 samples with the
// impulse at index 8 (support < 7 * 2^j + 1, so no wrap).  Over the region
// {|psi| > tau max |psi|} (Eq. 13) the |psi|-weighted centroid and covariance
// (Eq. 14) and the ridge weight w = sum |psi| g / (sum g^2 + lambda) (Eq. 17)
// follow; the centroid is reported relative to 2^j k_c (Eq. 12, exact on the
// grid).  The splat shape is the eigen-decomposition of the covariance.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "vbm_internal.h"

namespace vbm {

static std::vector<double> conv(const std::vector<double> &a, const std::vector<double> &b)
{
    std::vector<double> c(a.size() + b.size() - 1, 0.0);
    for (size_t i = 0; i < a.size(); i++)
        for (size_t j = 0; j < b.size(); j++) c[i + j] += a[i] * b[j];
    return c;
}

static std::map<int, double> centred(const std::vector<double> &v, double target_sum)
{
    // drop (near) zero end taps, centre, rescale
    size_t lo = 0, hi = v.size();
    while (lo < hi && std::fabs(v[lo]) < 1e-15) lo++;
    while (hi > lo && std::fabs(v[hi - 1]) < 1e-15) hi--;
    double s = 0.0;
    for (size_t i = lo; i < hi; i++) s += v[i];
    std::map<int, double> m;
    int half = (int)(hi - lo) / 2;
    for (size_t i = lo; i < hi; i++) m[(int)(i - lo) - half] = v[i] * target_sum / s;
    return m;
}

FilterBank make_filters(int wavelet)
{
    FilterBank fb;
    if (wavelet == 1) {
        const double s = 1.0 / std::sqrt(2.0);
        fb.ht = {{0, s}, {1, s}};
        fb.gt = {{-1, s}, {0, -s}};
        fb.h = {{0, s}, {1, s}};
        fb.g = {{-1, s}, {0, -s}};
        return fb;
    }
    // real root of 20x^3 + 10x^2 + 4x + 1 by bisection on [-1, 0] then Newton
    auto P = [](double x) { return ((20.0 * x + 10.0) * x + 4.0) * x + 1.0; };
    auto dP = [](double x) { return (60.0 * x + 20.0) * x + 4.0; };
    double lo = -1.0, hi = 0.0;
    for (int i = 0; i < 200; i++) {
        double mid = 0.5 * (lo + hi);
        if (P(mid) > 0) hi = mid; else lo = mid;
    }
    double xr = 0.5 * (lo + hi);
    for (int i = 0; i < 4; i++) xr -= P(xr) / dP(xr);
    // 20x^3 + 10x^2 + 4x + 1 = 20 (x - xr)(x^2 + p x + q)
    const double p = 0.5 + xr;
    const double q = 0.2 + p * xr;
    const std::vector<double> sin2 = {-0.25, 0.5, -0.25}, cos2 = {0.25, 0.5, 0.25}, one = {0.0, 1.0, 0.0};
    std::vector<double> cos4 = conv(cos2, cos2);
    std::vector<double> lin(3), quad(5, 0.0);
    for (int i = 0; i < 3; i++) lin[i] = one[i] - sin2[i] / xr;
    std::vector<double> s4 = conv(sin2, sin2);
    for (int i = 0; i < 5; i++) quad[i] = s4[i] / q;
    for (int i = 0; i < 3; i++) quad[i + 1] += (p * sin2[i] + q * one[i]) / q;
    fb.h = centred(conv(cos4, lin), std::sqrt(2.0));    // 7 taps: synthesis low-pass
    fb.ht = centred(conv(cos4, quad), std::sqrt(2.0));  // 9 taps: analysis low-pass
    for (auto &kv : fb.h) fb.gt[kv.first] = (kv.first % 2 ? -1.0 : 1.0) * kv.second;
    for (auto &kv : fb.ht) fb.g[kv.first] = (kv.first % 2 ? -1.0 : 1.0) * kv.second;
    return fb;
}

// 1D response of an impulse at index k of the level-j band (band 0 = low, 1 = high)
static std::vector<double> response_1d(const FilterBank &fb, int L, int j, int band, int k)
{
    std::vector<double> c(L, 0.0);
    c[band * (L >> j) + k] = 1.0;
    for (int lev = j; lev >= 1; lev--) {
        const int n = L >> (lev - 1), half = n / 2;
        std::vector<double> x(n, 0.0);
        for (int kk = 0; kk < half; kk++) {
            const double a = c[kk], d = c[half + kk];
            if (a != 0.0)
                for (auto &t : fb.h) x[(((2 * kk + t.first) % n) + n) % n] += t.second * a;
            if (d != 0.0)
                for (auto &t : fb.g) x[(((2 * kk + 1 + t.first) % n) + n) % n] += t.second * d;
        }
        std::copy(x.begin(), x.end(), c.begin());
    }
    return c;
}

// Cyclic Jacobi eigen-decomposition of a symmetric 3x3 matrix: A = V diag(e) V^T.
static void eig3(const double A_in[3][3], double e[3], double V[3][3])
{
    double A[3][3];
    std::memcpy(A, A_in, sizeof(A));
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) V[i][j] = i == j;
    for (int sweep = 0; sweep < 60; sweep++) {
        double off = std::fabs(A[0][1]) + std::fabs(A[0][2]) + std::fabs(A[1][2]);
        if (off < 1e-300) break;
        for (int p = 0; p < 2; p++)
            for (int q = p + 1; q < 3; q++) {
                if (A[p][q] == 0.0) continue;
                double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 3; k++) {
                    double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; k++) {
                    double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; k++) {
                    double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < 3; i++) e[i] = A[i][i];
}

static void rot_to_quat(const double R[3][3], double q[4])
{
    double tr = R[0][0] + R[1][1] + R[2][2];
    if (tr > 0) {
        double s = std::sqrt(tr + 1.0) * 2;
        q[0] = 0.25 * s; q[1] = (R[2][1] - R[1][2]) / s; q[2] = (R[0][2] - R[2][0]) / s; q[3] = (R[1][0] - R[0][1]) / s;
    } else if (R[0][0] > R[1][1] && R[0][0] > R[2][2]) {
        double s = std::sqrt(1.0 + R[0][0] - R[1][1] - R[2][2]) * 2;
        q[0] = (R[2][1] - R[1][2]) / s; q[1] = 0.25 * s; q[2] = (R[0][1] + R[1][0]) / s; q[3] = (R[0][2] + R[2][0]) / s;
    } else if (R[1][1] > R[2][2]) {
        double s = std::sqrt(1.0 + R[1][1] - R[0][0] - R[2][2]) * 2;
        q[0] = (R[0][2] - R[2][0]) / s; q[1] = (R[0][1] + R[1][0]) / s; q[2] = 0.25 * s; q[3] = (R[1][2] + R[2][1]) / s;
    } else {
        double s = std::sqrt(1.0 + R[2][2] - R[0][0] - R[1][1]) * 2;
        q[0] = (R[1][0] - R[0][1]) / s; q[1] = (R[0][2] + R[2][0]) / s; q[2] = (R[1][2] + R[2][1]) / s; q[3] = 0.25 * s;
    }
    double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; i++) q[i] /= n;
}

static void bank_entry(const FilterBank &fb, int wavelet, int j, const int o[3], double tau, double ridge_rel,
                       vbm_bank_entry *e)
{
    const int S = wavelet == 1 ? 4 : 16;
    const int L = (1 << j) * S, kc = S / 2;
    std::vector<double> r[3];
    int lo[3], hi[3];
    for (int d = 0; d < 3; d++) {
        r[d] = response_1d(fb, L, j, o[d], kc);
        lo[d] = L;
        hi[d] = -1;
        for (int i = 0; i < L; i++)
            if (r[d][i] != 0.0) { lo[d] = std::min(lo[d], i); hi[d] = std::max(hi[d], i); }
    }
    double mx = 0.0, total = 0.0;
    for (int z = lo[2]; z <= hi[2]; z++)
        for (int y = lo[1]; y <= hi[1]; y++)
            for (int x = lo[0]; x <= hi[0]; x++) {
                double m = std::fabs(r[0][x] * r[1][y] * r[2][z]);
                mx = std::max(mx, m);
                total += m;
            }
    // W = |psi| / total; ROI W > tau max W
    const double wmax = mx / total, thr = tau * wmax;
    double sw = 0.0, s1[3] = {0, 0, 0};
    for (int z = lo[2]; z <= hi[2]; z++)
        for (int y = lo[1]; y <= hi[1]; y++)
            for (int x = lo[0]; x <= hi[0]; x++) {
                double W = std::fabs(r[0][x] * r[1][y] * r[2][z]) / total;
                if (!(W > thr)) continue;
                sw += W;
                s1[0] += W * x; s1[1] += W * y; s1[2] += W * z;
            }
    double u[3] = {s1[0] / sw, s1[1] / sw, s1[2] / sw};
    double cov[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int z = lo[2]; z <= hi[2]; z++)
        for (int y = lo[1]; y <= hi[1]; y++)
            for (int x = lo[0]; x <= hi[0]; x++) {
                double W = std::fabs(r[0][x] * r[1][y] * r[2][z]) / total;
                if (!(W > thr)) continue;
                double dd[3] = {x - u[0], y - u[1], z - u[2]};
                for (int a = 0; a < 3; a++)
                    for (int b = 0; b < 3; b++) cov[a][b] += W * dd[a] * dd[b];
            }
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) cov[a][b] /= sw;
    // ridge weight over the ROI
    double det = cov[0][0] * (cov[1][1] * cov[2][2] - cov[1][2] * cov[2][1]) -
                 cov[0][1] * (cov[1][0] * cov[2][2] - cov[1][2] * cov[2][0]) +
                 cov[0][2] * (cov[1][0] * cov[2][1] - cov[1][1] * cov[2][0]);
    double inv[3][3];
    inv[0][0] = (cov[1][1] * cov[2][2] - cov[1][2] * cov[2][1]) / det;
    inv[0][1] = (cov[0][2] * cov[2][1] - cov[0][1] * cov[2][2]) / det;
    inv[0][2] = (cov[0][1] * cov[1][2] - cov[0][2] * cov[1][1]) / det;
    inv[1][0] = inv[0][1];
    inv[1][1] = (cov[0][0] * cov[2][2] - cov[0][2] * cov[2][0]) / det;
    inv[1][2] = (cov[0][2] * cov[1][0] - cov[0][0] * cov[1][2]) / det;
    inv[2][0] = inv[0][2];
    inv[2][1] = inv[1][2];
    inv[2][2] = (cov[0][0] * cov[1][1] - cov[0][1] * cov[1][0]) / det;
    double yg = 0.0, gg = 0.0;
    for (int z = lo[2]; z <= hi[2]; z++)
        for (int y = lo[1]; y <= hi[1]; y++)
            for (int x = lo[0]; x <= hi[0]; x++) {
                double Y = std::fabs(r[0][x] * r[1][y] * r[2][z]);
                if (!(Y / total > thr)) continue;
                double dd[3] = {x - u[0], y - u[1], z - u[2]};
                double qf = 0.0;
                for (int a = 0; a < 3; a++)
                    for (int b = 0; b < 3; b++) qf += dd[a] * inv[a][b] * dd[b];
                double G = std::exp(-0.5 * qf);
                yg += Y * G;
                gg += G * G;
            }
    e->j = j;
    for (int d = 0; d < 3; d++) {
        e->o[d] = o[d];
        e->u[d] = u[d] - (double)(1 << j) * kc;
    }
    e->cov[0] = cov[0][0]; e->cov[1] = cov[1][1]; e->cov[2] = cov[2][2];
    e->cov[3] = cov[0][1]; e->cov[4] = cov[0][2]; e->cov[5] = cov[1][2];
    e->w = yg / (gg + ridge_rel * gg);
    double off = std::max(std::fabs(cov[0][1]), std::max(std::fabs(cov[0][2]), std::fabs(cov[1][2])));
    double dmax = std::max(cov[0][0], std::max(cov[1][1], cov[2][2]));
    if (off <= 1e-9 * dmax) {
        for (int d = 0; d < 3; d++) e->log_scale[d] = (float)(0.5 * std::log(cov[d][d]));
        e->quat[0] = 1.f; e->quat[1] = e->quat[2] = e->quat[3] = 0.f;
    } else {
        double ev[3], V[3][3], q[4];
        eig3(cov, ev, V);
        double dV = V[0][0] * (V[1][1] * V[2][2] - V[1][2] * V[2][1]) - V[0][1] * (V[1][0] * V[2][2] - V[1][2] * V[2][0]) +
                    V[0][2] * (V[1][0] * V[2][1] - V[1][1] * V[2][0]);
        if (dV < 0)
            for (int k = 0; k < 3; k++) V[k][0] = -V[k][0];
        rot_to_quat(V, q);
        for (int d = 0; d < 3; d++) e->log_scale[d] = (float)(0.5 * std::log(ev[d]));
        for (int d = 0; d < 4; d++) e->quat[d] = (float)q[d];
    }
}

}  // namespace vbm

extern "C" vbm_status vbm_bank_build(int levels, int wavelet, double tau, double ridge_rel, vbm_bank *out)
{
    VBM_ARG(out, "null argument");
    VBM_ARG(levels >= 1 && levels <= 9 && 7 * levels + 1 <= 64, "levels must be in [1, 9]");
    VBM_ARG(wavelet == 0 || wavelet == 1, "wavelet must be 0 (bior4.4) or 1 (haar)");
    VBM_ARG(tau > 0.0 && tau < 1.0, "tau must be in (0, 1)");
    VBM_ARG(ridge_rel >= 0.0, "ridge_rel must be non-negative");
    std::memset(out, 0, sizeof(*out));
    out->levels = levels;
    out->wavelet = wavelet;
    out->tau = tau;
    out->ridge_rel = ridge_rel;
    vbm::FilterBank fb = vbm::make_filters(wavelet);
    int n = 0;
    for (int j = 1; j <= levels; j++)
        for (int code = 0; code < 8; code++) {
            if (code == 0 && j != levels) continue;
            int o[3] = {code & 1, (code >> 1) & 1, (code >> 2) & 1};
            vbm::bank_entry(fb, wavelet, j, o, tau, ridge_rel, &out->sub[n++]);
        }
    out->n_sub = n;
    return VBM_OK;
}

// Ablation variants of the bank (Sec. 5.4).  VBM_BANK_ISOTROPIC ("w/o
// transition bank"): every covariance becomes sigma_iso^2 I, sigma_iso the
// mean over the bank's subbands of det(Sigma_{j,o})^(1/6), the average
// spatial extent of the full bank; centres and weights are kept.
// VBM_BANK_UNIT_WEIGHT ("w/o energy projection"): every w_{j,o} = 1.
extern "C" vbm_status vbm_bank_ablate(vbm_bank *bank, int32_t flags)
{
    VBM_ARG(bank, "null argument");
    VBM_ARG(bank->n_sub >= 1 && bank->n_sub <= 64, "bank has no entries");
    VBM_ARG((flags & ~(VBM_BANK_ISOTROPIC | VBM_BANK_UNIT_WEIGHT)) == 0, "unknown ablation flag");
    if (flags & VBM_BANK_ISOTROPIC) {
        double mean = 0.0;
        for (int i = 0; i < bank->n_sub; i++) {
            const double *c = bank->sub[i].cov;   // xx yy zz xy xz yz
            const double det = c[0] * (c[1] * c[2] - c[5] * c[5]) - c[3] * (c[3] * c[2] - c[5] * c[4]) +
                               c[4] * (c[3] * c[5] - c[1] * c[4]);
            mean += std::pow(det, 1.0 / 6.0);
        }
        const double sigma = mean / bank->n_sub;
        for (int i = 0; i < bank->n_sub; i++) {
            vbm_bank_entry &e = bank->sub[i];
            e.cov[0] = e.cov[1] = e.cov[2] = sigma * sigma;
            e.cov[3] = e.cov[4] = e.cov[5] = 0.0;
            for (int d = 0; d < 3; d++) e.log_scale[d] = (float)std::log(sigma);
            e.quat[0] = 1.f;
            e.quat[1] = e.quat[2] = e.quat[3] = 0.f;
        }
    }
    if (flags & VBM_BANK_UNIT_WEIGHT)
        for (int i = 0; i < bank->n_sub; i++) bank->sub[i].w = 1.0;
    return VBM_OK;
}

