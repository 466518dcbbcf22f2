// Fourier-neural-operator surrogate: pulse parameters -> focal-region field.
//
// Network (per sample, patch P^3, width C):
//   v0 = W_lift [params, x, y, z] + b_lift                     (pointwise)
//   v_l = act( S_l(v_{l-1}) + W_l v_{l-1} + b_l ),  l = 1..L     (act = GELU, none on l = L)
//   out = W_q2 GELU(W_q1 v_L + b_q1) + b_q2
// S_l is the spectral convolution: truncated DFT of each channel to kx in
// [0, m) (half spectrum, real input) and ky, kz in {0..m-1, P-m..P-1}, a complex
// C x C matrix per kept mode, and the inverse (real output, kx > 0 counted twice).
//
// Every dense contraction is a call of the tensor-core GEMM (gemm.cu): the
// truncated DFTs contract the last axis of their input and write the new
// spectral axis first, so each stage is one strided GEMM per real/imaginary
// part.  All stages are real-linear in the stored (re, im) arrays, so each
// backward stage is the same GEMM with the transposed real matrix.  The
// per-mode complex mixing, GELU, the bias sums, the MSE loss and Adam are small
// elementwise / reduction kernels.  Tensors are float32; GEMM tiles are rounded
// to bfloat16 (float32 accumulation).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <random>
#include <string>
#include <vector>

#include "../../include/psatd.h"
#include "common.cuh"

namespace psatd {



namespace {

constexpr double kPi = 3.14159265358979323846;

// ------------------------------------------------------------ small kernels
__global__ void features_kernel(const float* __restrict__ prm, int np, int B, int P, float* __restrict__ feat) {
    const long long nv = (long long)P * P * P;
    const int nch = np + 3;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)B * nch * nv;
         e += (long long)gridDim.x * blockDim.x) {
        const long long vox = e % nv;
        const int ch = (int)((e / nv) % nch);
        const int b = (int)(e / (nv * nch));
        float v;
        if (ch < np) v = prm[b * np + ch];
        else {
            const int x = (int)(vox % P), y = (int)((vox / P) % P), z = (int)(vox / ((long long)P * P));
            const int q = ch == np ? x : (ch == np + 1 ? y : z);
            v = -1.f + 2.f * q / P;
        }
        feat[e] = v;
    }
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
    return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// z[b][c][v] += bias[c]; a = act(z) (act = GELU if gelu else identity); a may be z
__global__ void bias_act_kernel(float* z, float* a, const float* __restrict__ bias,
                                int B, int C, long long nv, int use_gelu) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)B * C * nv;
         e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)((e / nv) % C);
        const float v = z[e] + bias[c];
        z[e] = v;
        a[e] = use_gelu ? gelu(v) : v;
    }
}

// g_z = g_a * act'(z); g_z may be g_a
__global__ void act_back_kernel(const float* __restrict__ z, const float* ga, float* gz,
                                long long n, int use_gelu) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        gz[e] = use_gelu ? ga[e] * gelu_grad(z[e]) : ga[e];
}

// gbias[c] = sum over b, v of g[b][c][v]   (one block per channel)
__global__ void bias_grad_kernel(const float* __restrict__ g, float* __restrict__ gbias, int B, int C, long long nv) {
    const int c = blockIdx.x;
    double s = 0.0;
    for (int b = 0; b < B; ++b) {
        const float* row = g + ((long long)b * C + c) * nv;
        for (long long v = threadIdx.x; v < nv; v += blockDim.x) s += row[v];
    }
    __shared__ double sh[256];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) gbias[c] = (float)sh[0];
}

// Per-mode complex mixing.  Spectra laid out [part][mode][b][ch]; weights
// R[part][mode][i][o].  U[mode][b][o] = sum_i V[mode][b][i] R[mode][i][o].
__global__ void mix_fwd_kernel(const float* __restrict__ V, const float* __restrict__ R, float* __restrict__ U,
                               int modes, int B, int C) {
    const long long per = (long long)modes * B * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < per; e += (long long)gridDim.x * blockDim.x) {
        const int o = (int)(e % C);
        const long long mb = e / C;                      // mode * B + b
        const int mode = (int)(mb / B);
        const float* vr = V + mb * C;
        const float* vi = V + per + mb * C;
        const float* rr = R + (long long)mode * C * C + o;
        const float* ri = R + (long long)modes * C * C + (long long)mode * C * C + o;
        float ur = 0.f, ui = 0.f;
        for (int i = 0; i < C; ++i) {
            const float a = vr[i], b = vi[i], c = rr[i * C], d = ri[i * C];
            ur += a * c - b * d;
            ui += a * d + b * c;
        }
        U[e] = ur;
        U[per + e] = ui;
    }
}

// gV[mode][b][i] = sum_o (gUr R_r + gUi R_i, -gUr R_i + gUi R_r)
__global__ void mix_back_input_kernel(const float* __restrict__ gU, const float* __restrict__ R, float* __restrict__ gV,
                                      int modes, int B, int C) {
    const long long per = (long long)modes * B * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < per; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % C);
        const long long mb = e / C;
        const int mode = (int)(mb / B);
        const float* gr = gU + mb * C;
        const float* gi = gU + per + mb * C;
        const float* rr = R + (long long)mode * C * C + (long long)i * C;
        const float* ri = R + (long long)modes * C * C + (long long)mode * C * C + (long long)i * C;
        float vr = 0.f, vi = 0.f;
        for (int o = 0; o < C; ++o) {
            vr += gr[o] * rr[o] + gi[o] * ri[o];
            vi += -gr[o] * ri[o] + gi[o] * rr[o];
        }
        gV[e] = vr;
        gV[per + e] = vi;
    }
}

// gR[mode][i][o] = sum_b (gUr Vr + gUi Vi, -gUr Vi + gUi Vr)
__global__ void mix_back_weight_kernel(const float* __restrict__ gU, const float* __restrict__ V, float* __restrict__ gR,
                                       int modes, int B, int C) {
    const long long per = (long long)modes * B * C;
    const long long nw = (long long)modes * C * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nw; e += (long long)gridDim.x * blockDim.x) {
        const int o = (int)(e % C);
        const int i = (int)((e / C) % C);
        const int mode = (int)(e / ((long long)C * C));
        float sr = 0.f, si = 0.f;
        for (int b = 0; b < B; ++b) {
            const long long base = ((long long)mode * B + b) * C;
            const float gr = gU[base + o], gi = gU[per + base + o];
            const float vr = V[base + i], vi = V[per + base + i];
            sr += gr * vr + gi * vi;
            si += -gr * vi + gi * vr;
        }
        gR[e] = sr;
        gR[nw + e] = si;
    }
}

// loss partials of mean((y - t)^2) and g = 2 (y - t) / n
__global__ void mse_kernel(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ g, long long n,
                           double* __restrict__ partial) {
    double s = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float d = y[e] - t[e];
        s += (double)d * d;
        g[e] = 2.f * d / (float)n;
    }
    __shared__ double sh[256];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                            long long n, float lr, float b1, float b2, float eps, float wd, float c1, float c2) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float gr = g[e] + wd * p[e];
        const float mm = b1 * m[e] + (1.f - b1) * gr;
        const float vv = b2 * v[e] + (1.f - b2) * gr * gr;
        m[e] = mm;
        v[e] = vv;
        p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    }
}

int grid_for(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 152 * 32 ? (b < 1 ? 1 : b) : 152 * 32);
}

}  // namespace

}  // namespace psatd

using namespace psatd;

struct psatd_fno {
    psatd_fno_config cfg{};
    cudaStream_t stream = nullptr;
    int P = 0, C = 0, L = 0, m = 0, NT = 0, MODES = 0, H = 0, NO = 0, NP = 0, maxB = 0;
    long long NV = 0;
    // parameters, gradients, Adam moments (flat)
    float *par = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
    long long npar = 0;
    long long o_lift_w, o_lift_b, o_q1_w, o_q1_b, o_q2_w, o_q2_b;
    std::vector<long long> o_R, o_W, o_b;
    // DFT matrices
    float *Fx = nullptr, *By1 = nullptr, *By2 = nullptr, *Bz1 = nullptr, *Bz2 = nullptr, *Bx1 = nullptr, *Bx2 = nullptr;
    // activations (per layer): input a_l, pre-activation z_l, spectral intermediates
    std::vector<float*> act, pre, T1, T2, T3, U3, W1, W2;
    float *feat = nullptr, *hq = nullptr, *zq = nullptr, *out = nullptr, *gbuf0 = nullptr, *gbuf1 = nullptr;
    float *gT = nullptr, *gT2 = nullptr, *gout = nullptr;
    double* partial = nullptr;
    int adam_t = 0;
    std::string err = "no error";
};

namespace {

psatd_status fno_fail(psatd_fno* f, psatd_status s, const std::string& m) {
    if (f) f->err = m;
    return s;
}

#define FCK(call)                                                                                 \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return fno_fail(f, PSATD_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

// C(m,n) = A(m,k) B(k,n), 1-level batch
GemmArgs G(int M, int N, int K, const float* A, long long sAm, long long sAk, const float* B, long long sBk,
           long long sBn, float* C, long long sCm, long long sCn, float beta, int nb = 1, long long sAb = 0,
           long long sBb = 0, long long sCb = 0) {
    GemmArgs g{};
    g.M = M; g.N = N; g.K = K; g.nb0 = nb; g.nb1 = 1;
    g.A = A; g.sAb0 = sAb; g.sAm = sAm; g.sAk = sAk;
    g.B = B; g.sBb0 = sBb; g.sBk = sBk; g.sBn = sBn;
    g.C = C; g.sCb0 = sCb; g.sCm = sCm; g.sCn = sCn;
    g.alpha = 1.f; g.beta = beta; g.ksplit = 1;
    return g;
}

int freq_t(int j, int m, int P) { return j < m ? j : P - 2 * m + j; }

}  // namespace

extern "C" {

psatd_status psatd_fno_create(const psatd_fno_config* cfg, unsigned long long seed, void* stream, psatd_fno** out) {
    if (!cfg || !out) return PSATD_ERR_ARG;
    *out = nullptr;
    const int P = cfg->patch, C = cfg->width, L = cfg->layers, m = cfg->modes;
    if (P < 4 || P > 128 || (P & 1) || C < 1 || C > 256 || L < 1 || L > 16 || m < 1 || 2 * m > P ||
        cfg->in_params < 0 || cfg->in_params > 64 || cfg->hidden < 1 || cfg->out_channels < 1 || cfg->max_batch < 1)
        return PSATD_ERR_ARG;
    psatd_fno* f = new (std::nothrow) psatd_fno();
    if (!f) return PSATD_ERR_OOM;
    f->cfg = *cfg;
    f->stream = static_cast<cudaStream_t>(stream);
    f->P = P; f->C = C; f->L = L; f->m = m; f->NT = 2 * m; f->MODES = m * 4 * m * m;
    f->H = cfg->hidden; f->NO = cfg->out_channels; f->NP = cfg->in_params; f->maxB = cfg->max_batch;
    f->NV = (long long)P * P * P;
    const int FI = f->NP + 3;
    // parameter layout
    long long o = 0;
    f->o_lift_w = o; o += (long long)C * FI;
    f->o_lift_b = o; o += C;
    for (int l = 0; l < L; ++l) {
        f->o_R.push_back(o); o += 2LL * f->MODES * C * C;
        f->o_W.push_back(o); o += (long long)C * C;
        f->o_b.push_back(o); o += C;
    }
    f->o_q1_w = o; o += (long long)f->H * C;
    f->o_q1_b = o; o += f->H;
    f->o_q2_w = o; o += (long long)f->NO * f->H;
    f->o_q2_b = o; o += f->NO;
    f->npar = o;
    // host init: uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) for pointwise, scale/(C*C) * U[0,1) spectral
    std::vector<float> h((size_t)o, 0.f);
    std::mt19937_64 rng(seed);
    std::uniform_real_distribution<double> U(0.0, 1.0);
    auto fill = [&](long long off, long long n, double lo, double hi) {
        for (long long i = 0; i < n; ++i) h[off + i] = (float)(lo + (hi - lo) * U(rng));
    };
    fill(f->o_lift_w, (long long)C * FI, -1.0 / std::sqrt(FI), 1.0 / std::sqrt(FI));
    for (int l = 0; l < L; ++l) {
        fill(f->o_R[l], 2LL * f->MODES * C * C, 0.0, 1.0 / ((double)C * C));
        fill(f->o_W[l], (long long)C * C, -1.0 / std::sqrt(C), 1.0 / std::sqrt(C));
    }
    fill(f->o_q1_w, (long long)f->H * C, -1.0 / std::sqrt(C), 1.0 / std::sqrt(C));
    fill(f->o_q2_w, (long long)f->NO * f->H, -1.0 / std::sqrt(f->H), 1.0 / std::sqrt(f->H));

    auto alloc = [&](float** p, long long n) -> bool {
        return cudaMalloc(p, (size_t)n * sizeof(float)) == cudaSuccess;
    };
    bool ok = alloc(&f->par, o) && alloc(&f->grad, o) && alloc(&f->m1, o) && alloc(&f->m2, o);
    // DFT matrices (float64 on the host, rounded once)
    const int NT = f->NT;
    std::vector<float> fx((size_t)P * 2 * m), by1((size_t)P * 2 * NT), by2((size_t)P * 2 * NT),
        bx1((size_t)m * P), bx2((size_t)m * P), bz1((size_t)NT * 2 * P), bz2((size_t)NT * 2 * P);
    for (int x = 0; x < P; ++x)
        for (int k = 0; k < m; ++k) {
            const double th = 2 * kPi * k * x / P;
            fx[(size_t)x * 2 * m + k] = (float)std::cos(th);
            fx[(size_t)x * 2 * m + m + k] = (float)(-std::sin(th));
        }
    // forward complex stage: out = re * [Cs | -Sn] + im * [Sn | Cs]  (kernel exp(-i th))
    for (int y = 0; y < P; ++y)
        for (int j = 0; j < NT; ++j) {
            const double th = 2 * kPi * freq_t(j, m, P) * y / P;
            by1[(size_t)y * 2 * NT + j] = (float)std::cos(th);
            by1[(size_t)y * 2 * NT + NT + j] = (float)(-std::sin(th));
            by2[(size_t)y * 2 * NT + j] = (float)std::sin(th);
            by2[(size_t)y * 2 * NT + NT + j] = (float)std::cos(th);
        }
    // inverse complex stage: out = re * [Cs | Sn] + im * [-Sn | Cs]  (kernel exp(+i th))
    for (int j = 0; j < NT; ++j)
        for (int z = 0; z < P; ++z) {
            const double th = 2 * kPi * freq_t(j, m, P) * z / P;
            bz1[(size_t)j * 2 * P + z] = (float)std::cos(th);
            bz1[(size_t)j * 2 * P + P + z] = (float)std::sin(th);
            bz2[(size_t)j * 2 * P + z] = (float)(-std::sin(th));
            bz2[(size_t)j * 2 * P + P + z] = (float)std::cos(th);
        }
    // inverse x: u = (1/P^3) sum_k w_k (re cos - im sin), w_0 = 1, w_k = 2
    const double inv = 1.0 / ((double)P * P * P);
    for (int k = 0; k < m; ++k)
        for (int x = 0; x < P; ++x) {
            const double th = 2 * kPi * k * x / P, w = (k == 0 ? 1.0 : 2.0) * inv;
            bx1[(size_t)k * P + x] = (float)(w * std::cos(th));
            bx2[(size_t)k * P + x] = (float)(-w * std::sin(th));
        }
    ok = ok && alloc(&f->Fx, fx.size()) && alloc(&f->By1, by1.size()) && alloc(&f->By2, by2.size()) &&
         alloc(&f->Bz1, bz1.size()) && alloc(&f->Bz2, bz2.size()) && alloc(&f->Bx1, bx1.size()) &&
         alloc(&f->Bx2, bx2.size());
    // activations for max batch
    const long long B = f->maxB, NV = f->NV;
    const long long nT1 = 2LL * m * B * C * P * P, nT2 = 2LL * NT * m * B * C * P, nT3 = 2LL * f->MODES * B * C;
    const long long nW1 = 2LL * P * NT * m * B * C, nW2 = 2LL * P * P * m * B * C;
    for (int l = 0; l <= L && ok; ++l) {
        float *a = nullptr, *z = nullptr;
        ok = alloc(&a, B * C * NV) && alloc(&z, B * C * NV);
        f->act.push_back(a);
        f->pre.push_back(z);
    }
    for (int l = 0; l < L && ok; ++l) {
        float *t1, *t2, *t3, *u3, *w1, *w2;
        ok = alloc(&t1, nT1) && alloc(&t2, nT2) && alloc(&t3, nT3) && alloc(&u3, nT3) && alloc(&w1, nW1) && alloc(&w2, nW2);
        if (!ok) break;
        f->T1.push_back(t1); f->T2.push_back(t2); f->T3.push_back(t3); f->U3.push_back(u3);
        f->W1.push_back(w1); f->W2.push_back(w2);
    }
    long long big = std::max(std::max(nT1, nW2), B * C * NV);
    ok = ok && alloc(&f->feat, B * FI * NV) && alloc(&f->hq, B * f->H * NV) && alloc(&f->zq, B * f->H * NV) &&
         alloc(&f->out, B * f->NO * NV) && alloc(&f->gbuf0, std::max(B * f->H * NV, big)) &&
         alloc(&f->gbuf1, std::max(B * f->H * NV, big)) && alloc(&f->gT, std::max(big, nW1)) &&
         alloc(&f->gT2, std::max(big, nW1)) && alloc(&f->gout, B * f->NO * NV);
    ok = ok && cudaMalloc(&f->partial, 4096 * sizeof(double)) == cudaSuccess;
    if (!ok) {
        psatd_fno_destroy(f);
        return PSATD_ERR_OOM;
    }
    cudaStream_t s = f->stream;
    bool cp = cudaMemcpyAsync(f->par, h.data(), (size_t)o * sizeof(float), cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaMemsetAsync(f->m1, 0, (size_t)o * sizeof(float), s) == cudaSuccess &&
              cudaMemsetAsync(f->m2, 0, (size_t)o * sizeof(float), s) == cudaSuccess &&
              cudaMemcpyAsync(f->Fx, fx.data(), fx.size() * 4, cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(f->By1, by1.data(), by1.size() * 4, cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(f->By2, by2.data(), by2.size() * 4, cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(f->Bz1, bz1.data(), bz1.size() * 4, cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(f->Bz2, bz2.data(), bz2.size() * 4, cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(f->Bx1, bx1.data(), bx1.size() * 4, cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(f->Bx2, bx2.data(), bx2.size() * 4, cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaStreamSynchronize(s) == cudaSuccess;
    if (!cp) {
        psatd_fno_destroy(f);
        return PSATD_ERR_CUDA;
    }
    *out = f;
    return PSATD_OK;
}

void psatd_fno_destroy(psatd_fno* f) {
    if (!f) return;
    if (f->stream) cudaStreamSynchronize(f->stream);
    float* ps[] = {f->par, f->grad, f->m1, f->m2, f->Fx, f->By1, f->By2, f->Bz1, f->Bz2, f->Bx1, f->Bx2,
                   f->feat, f->hq, f->zq, f->out, f->gbuf0, f->gbuf1, f->gT, f->gT2, f->gout};
    for (float* p : ps)
        if (p) cudaFree(p);
    for (auto* v : {&f->act, &f->pre, &f->T1, &f->T2, &f->T3, &f->U3, &f->W1, &f->W2})
        for (float* p : *v)
            if (p) cudaFree(p);
    if (f->partial) cudaFree(f->partial);
    delete f;
}

long long psatd_fno_num_params(const psatd_fno* f) { return f ? f->npar : 0; }

psatd_status psatd_fno_buffers(psatd_fno* f, float** params, float** grads, float** output) {
    if (!f) return PSATD_ERR_ARG;
    if (params) *params = f->par;
    if (grads) *grads = f->grad;
    if (output) *output = f->out;
    return PSATD_OK;
}

const char* psatd_fno_last_error(const psatd_fno* f) { return f ? f->err.c_str() : "NULL model"; }

}  // extern "C"

namespace {

// forward pass; leaves activations for the backward pass
psatd_status fno_forward(psatd_fno* f, const float* prm, int B) {
    const int P = f->P, C = f->C, m = f->m, NT = f->NT, FI = f->NP + 3;
    const long long NV = f->NV;
    cudaStream_t s = f->stream;
    features_kernel<<<grid_for(B * FI * NV), 256, 0, s>>>(prm, f->NP, B, P, f->feat);
    // lift: pre0[b] = W_lift (C x FI) feat[b] (FI x NV)
    FCK(launch_gemm(G(C, (int)NV, FI, f->par + f->o_lift_w, FI, 1, f->feat, NV, 1, f->pre[0], NV, 1, 0.f, B, 0,
                      FI * NV, C * NV), s));
    bias_act_kernel<<<grid_for(B * C * NV), 256, 0, s>>>(f->pre[0], f->act[0], f->par + f->o_lift_b, B, C, NV, 0);
    for (int l = 0; l < f->L; ++l) {
        const float* v = f->act[l];
        float* z = f->pre[l + 1];
        const long long M1 = (long long)B * C * P * P;          // rows (b,c,z,y)
        // X: T1[(part,kx)][(b,c,z,y)] = v[(b,c,z,y)][x] Fx[x][(part,kx)]
        FCK(launch_gemm(G((int)M1, 2 * m, P, v, P, 1, f->Fx, 2 * m, 1, f->T1[l], 1, M1, 0.f), s));
        // Y: rows (kx,b,c,z) per part, contract y; out [(part,ky)][rows]
        const long long Mh = (long long)m * B * C * P;
        FCK(launch_gemm(G((int)Mh, 2 * NT, P, f->T1[l], P, 1, f->By1, 2 * NT, 1, f->T2[l], 1, Mh, 0.f), s));
        FCK(launch_gemm(G((int)Mh, 2 * NT, P, f->T1[l] + Mh * P, P, 1, f->By2, 2 * NT, 1, f->T2[l], 1, Mh, 1.f), s));
        // Z: rows (ky,kx,b,c) per part, contract z
        const long long Mz = (long long)NT * m * B * C;
        FCK(launch_gemm(G((int)Mz, 2 * NT, P, f->T2[l], P, 1, f->By1, 2 * NT, 1, f->T3[l], 1, Mz, 0.f), s));
        FCK(launch_gemm(G((int)Mz, 2 * NT, P, f->T2[l] + Mz * P, P, 1, f->By2, 2 * NT, 1, f->T3[l], 1, Mz, 1.f), s));
        // mode mixing: T3 = [part][kz][ky][kx][b][c] = [part][mode][b][c]
        mix_fwd_kernel<<<grid_for((long long)f->MODES * B * C), 256, 0, s>>>(f->T3[l], f->par + f->o_R[l], f->U3[l],
                                                                            f->MODES, B, C);
        // Zi: rows r = (ky,kx,b,o), K = kz (stride Mz); out W1[(part,z)][r]
        FCK(launch_gemm(G((int)Mz, 2 * P, NT, f->U3[l], 1, Mz, f->Bz1, 2 * P, 1, f->W1[l], 1, Mz, 0.f), s));
        FCK(launch_gemm(G((int)Mz, 2 * P, NT, f->U3[l] + (long long)NT * Mz, 1, Mz, f->Bz2, 2 * P, 1, f->W1[l], 1, Mz, 1.f), s));
        // Yi: W1[part][z][ky][Q], Q = (kx,b,o); batch z, rows Q, K = ky; out W2[(part,y)][z][Q]
        const long long Q = (long long)m * B * C;
        FCK(launch_gemm(G((int)Q, 2 * P, NT, f->W1[l], 1, Q, f->Bz1, 2 * P, 1, f->W2[l], 1, (long long)P * Q, 0.f, P,
                          (long long)NT * Q, 0, Q), s));
        FCK(launch_gemm(G((int)Q, 2 * P, NT, f->W1[l] + (long long)P * NT * Q, 1, Q, f->Bz2, 2 * P, 1, f->W2[l], 1,
                          (long long)P * Q, 1.f, P, (long long)NT * Q, 0, Q), s));
        // Xi: W2[part][y][z][kx][(b,o)]; batch (y, z), rows (b,o), K = kx; out z[(b,o)][z][y][x]
        {
            GemmArgs g = G(B * C, P, m, f->W2[l], 1, (long long)B * C, f->Bx1, P, 1, z, NV, 1, 0.f);
            g.nb0 = P; g.nb1 = P;
            g.sAb0 = (long long)P * Q; g.sAb1 = Q;               // y, z
            g.sCb0 = P; g.sCb1 = (long long)P * P;
            FCK(launch_gemm(g, s));
            g.A = f->W2[l] + (long long)P * P * Q;
            g.B = f->Bx2;
            g.beta = 1.f;
            FCK(launch_gemm(g, s));
        }
        // pointwise W v added: z[b] += W (C x C) v[b]
        FCK(launch_gemm(G(C, (int)NV, C, f->par + f->o_W[l], C, 1, v, NV, 1, z, NV, 1, 1.f, B, 0, C * NV, C * NV), s));
        bias_act_kernel<<<grid_for(B * C * NV), 256, 0, s>>>(z, f->act[l + 1], f->par + f->o_b[l], B, C, NV,
                                                            l + 1 < f->L ? 1 : 0);
    }
    // projection
    const int H = f->H, NO = f->NO;
    FCK(launch_gemm(G(H, (int)NV, C, f->par + f->o_q1_w, C, 1, f->act[f->L], NV, 1, f->zq, NV, 1, 0.f, B, 0, C * NV,
                      H * NV), s));
    bias_act_kernel<<<grid_for(B * H * NV), 256, 0, s>>>(f->zq, f->hq, f->par + f->o_q1_b, B, H, NV, 1);
    FCK(launch_gemm(G(NO, (int)NV, H, f->par + f->o_q2_w, H, 1, f->hq, NV, 1, f->out, NV, 1, 0.f, B, 0, H * NV,
                      NO * NV), s));
    // bias only (no activation): out += b, in place
    bias_act_kernel<<<grid_for(B * NO * NV), 256, 0, s>>>(f->out, f->out, f->par + f->o_q2_b, B, NO, NV, 0);
    FCK(cudaGetLastError());
    return PSATD_OK;
}

// weight gradient gW (Mo x Ni) = sum_b gZ[b] (Mo x NV) * X[b]^T (NV x Ni), split over NV
cudaError_t weight_grad(psatd_fno* f, int Mo, int Ni, const float* gZ, const float* X, float* gW, int B) {
    for (int b = 0; b < B; ++b) {
        GemmArgs g = G(Mo, Ni, (int)f->NV, gZ + (long long)b * Mo * f->NV, f->NV, 1, X + (long long)b * Ni * f->NV, 1,
                       f->NV, gW, Ni, 1, b == 0 ? 0.f : 1.f);
        g.ksplit = (int)std::min<long long>(256, (f->NV + 4095) / 4096);
        cudaError_t e = launch_gemm(g, f->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

psatd_status fno_backward(psatd_fno* f, int B) {
    const int P = f->P, C = f->C, m = f->m, NT = f->NT, H = f->H, NO = f->NO, FI = f->NP + 3;
    const long long NV = f->NV;
    cudaStream_t s = f->stream;
    float* g = f->grad;
    // output layer: gout holds dL/dout
    bias_grad_kernel<<<NO, 256, 0, s>>>(f->gout, g + f->o_q2_b, B, NO, NV);
    FCK(weight_grad(f, NO, H, f->gout, f->hq, g + f->o_q2_w, B));
    // g_h = Wq2^T gout ; g_zq = g_h * gelu'(zq)
    FCK(launch_gemm(G(H, (int)NV, NO, f->par + f->o_q2_w, 1, H, f->gout, NV, 1, f->gbuf0, NV, 1, 0.f, B, 0, NO * NV,
                      H * NV), s));
    act_back_kernel<<<grid_for(B * H * NV), 256, 0, s>>>(f->zq, f->gbuf0, f->gbuf0, B * H * NV, 1);
    bias_grad_kernel<<<H, 256, 0, s>>>(f->gbuf0, g + f->o_q1_b, B, H, NV);
    FCK(weight_grad(f, H, C, f->gbuf0, f->act[f->L], g + f->o_q1_w, B));
    // g_a(L) = Wq1^T g_zq
    float* ga = f->gbuf1;
    FCK(launch_gemm(G(C, (int)NV, H, f->par + f->o_q1_w, 1, C, f->gbuf0, NV, 1, ga, NV, 1, 0.f, B, 0, H * NV, C * NV), s));
    for (int l = f->L - 1; l >= 0; --l) {
        // g_z = g_a * act'(z)
        float* gz = f->gbuf0;
        act_back_kernel<<<grid_for(B * C * NV), 256, 0, s>>>(f->pre[l + 1], ga, gz, B * C * NV, l + 1 < f->L ? 1 : 0);
        bias_grad_kernel<<<C, 256, 0, s>>>(gz, g + f->o_b[l], B, C, NV);
        FCK(weight_grad(f, C, C, gz, f->act[l], g + f->o_W[l], B));
        // g_v (pointwise part) = W^T g_z -> ga (act[l] gradient), overwritten
        FCK(launch_gemm(G(C, (int)NV, C, f->par + f->o_W[l], 1, C, gz, NV, 1, ga, NV, 1, 0.f, B, 0, C * NV, C * NV), s));
        // spectral part, adjoint of Xi: g_W2[part] = gz (rows (b,o), per (y,z): x) * Bx^T
        const long long Q = (long long)m * B * C, Mz = (long long)NT * m * B * C, Mh = (long long)m * B * C * P;
        float* gW2 = f->gT;        // layout of W2
        {
            GemmArgs a = G(B * C, m, P, gz, NV, 1, f->Bx1, 1, P, gW2, 1, (long long)B * C, 0.f);
            a.nb0 = P; a.nb1 = P;
            a.sAb0 = P; a.sAb1 = (long long)P * P;              // gz[(b,o)][z][y][x]: y stride P, z stride P^2
            a.sCb0 = (long long)P * Q; a.sCb1 = Q;
            FCK(launch_gemm(a, s));
            a.B = f->Bx2;
            a.C = gW2 + (long long)P * P * Q;
            FCK(launch_gemm(a, s));
        }
        // adjoint of Yi: g_W1[part'] = sum over (part, y) of gW2 rows; W2 = W1re*Bz1 + W1im*Bz2
        float* gW1 = f->gT2;
        for (int part = 0; part < 2; ++part) {
            GemmArgs a = G((int)Q, NT, 2 * P, gW2, 1, (long long)P * Q, part == 0 ? f->Bz1 : f->Bz2, 1, 2 * P,
                           gW1 + (long long)part * P * NT * Q, 1, Q, 0.f, P, Q, 0, (long long)NT * Q);
            FCK(launch_gemm(a, s));
        }
        // adjoint of Zi: g_U[part'] rows (ky,kx,b,o), K over (part,z) of gW1
        float* gU = f->gT;
        for (int part = 0; part < 2; ++part)
            FCK(launch_gemm(G((int)Mz, NT, 2 * P, gW1, 1, Mz, part == 0 ? f->Bz1 : f->Bz2, 1, 2 * P,
                              gU + (long long)part * NT * Mz, 1, Mz, 0.f), s));
        // mixing: weights and spectra
        mix_back_weight_kernel<<<grid_for((long long)f->MODES * C * C), 256, 0, s>>>(gU, f->T3[l], g + f->o_R[l], f->MODES, B, C);
        float* gV = f->gT2;
        mix_back_input_kernel<<<grid_for((long long)f->MODES * B * C), 256, 0, s>>>(gU, f->par + f->o_R[l], gV, f->MODES, B, C);
        // adjoint of Z: g_T2[part] (rows (ky,kx,b,c), K = z) = gV (rows, 2NT) * By_part^T
        float* gT2 = f->gT;
        for (int part = 0; part < 2; ++part)
            FCK(launch_gemm(G((int)Mz, P, 2 * NT, gV, 1, Mz, part == 0 ? f->By1 : f->By2, 1, 2 * NT,
                              gT2 + (long long)part * Mz * P, P, 1, 0.f), s));
        // adjoint of Y: g_T1[part] (rows (kx,b,c,z), K = y)
        float* gT1 = f->gT2;
        for (int part = 0; part < 2; ++part)
            FCK(launch_gemm(G((int)Mh, P, 2 * NT, gT2, 1, Mh, part == 0 ? f->By1 : f->By2, 1, 2 * NT,
                              gT1 + (long long)part * Mh * P, P, 1, 0.f), s));
        // adjoint of X: g_v += gT1 (rows (b,c,z,y), 2m) * Fx^T
        const long long M1 = (long long)B * C * P * P;
        FCK(launch_gemm(G((int)M1, P, 2 * m, gT1, 1, M1, f->Fx, 1, 2 * m, ga, P, 1, 1.f), s));
    }
    // lift
    float* gz = f->gbuf0;
    act_back_kernel<<<grid_for(B * C * NV), 256, 0, s>>>(f->pre[0], ga, gz, B * C * NV, 0);
    bias_grad_kernel<<<C, 256, 0, s>>>(gz, g + f->o_lift_b, B, C, NV);
    FCK(weight_grad(f, C, FI, gz, f->feat, g + f->o_lift_w, B));
    FCK(cudaGetLastError());
    return PSATD_OK;
}

}  // namespace

extern "C" {

psatd_status psatd_fno_forward(psatd_fno* f, const float* params_dev, int batch, float* out_dev) {
    if (!f || !params_dev || batch < 1 || batch > f->maxB) return fno_fail(f, PSATD_ERR_ARG, "bad arguments");
    psatd_status st = fno_forward(f, params_dev, batch);
    if (st) return st;
    if (out_dev && out_dev != f->out) {
        FCK(cudaMemcpyAsync(out_dev, f->out, (size_t)batch * f->NO * f->NV * sizeof(float), cudaMemcpyDeviceToDevice,
                            f->stream));
    }
    return PSATD_OK;
}

psatd_status psatd_fno_loss_backward(psatd_fno* f, const float* params_dev, int batch, const float* target_dev,
                                     double* loss) {
    if (!f || !params_dev || !target_dev || batch < 1 || batch > f->maxB)
        return fno_fail(f, PSATD_ERR_ARG, "bad arguments");
    psatd_status st = fno_forward(f, params_dev, batch);
    if (st) return st;
    const long long n = (long long)batch * f->NO * f->NV;
    const int nb = std::min(4096, grid_for(n));
    mse_kernel<<<nb, 256, 0, f->stream>>>(f->out, target_dev, f->gout, n, f->partial);
    st = fno_backward(f, batch);
    if (st) return st;
    if (loss) {
        std::vector<double> h(nb);
        FCK(cudaMemcpyAsync(h.data(), f->partial, nb * sizeof(double), cudaMemcpyDeviceToHost, f->stream));
        FCK(cudaStreamSynchronize(f->stream));
        double s = 0;
        for (double v : h) s += v;
        *loss = s / (double)n;
    }
    return PSATD_OK;
}

psatd_status psatd_fno_adam_step(psatd_fno* f, float lr, float beta1, float beta2, float eps, float weight_decay) {
    if (!f) return PSATD_ERR_ARG;
    f->adam_t += 1;
    const float c1 = 1.f - std::pow(beta1, (float)f->adam_t), c2 = 1.f - std::pow(beta2, (float)f->adam_t);
    adam_kernel<<<grid_for(f->npar), 256, 0, f->stream>>>(f->par, f->grad, f->m1, f->m2, f->npar, lr, beta1, beta2, eps,
                                                           weight_decay, c1, c2);
    FCK(cudaGetLastError());
    return PSATD_OK;
}

psatd_status psatd_gemm_bf16(int M, int N, int K, const float* A, long long sAm, long long sAk, const float* B,
                             long long sBk, long long sBn, float* C, long long sCm, long long sCn, float alpha,
                             float beta, int ksplit, void* cuda_stream) {
    if (!A || !B || !C || M < 0 || N < 0 || K < 0) return PSATD_ERR_ARG;
    GemmArgs g = G(M, N, K, A, sAm, sAk, B, sBk, sBn, C, sCm, sCn, beta);
    g.alpha = alpha;
    g.ksplit = ksplit < 1 ? 1 : ksplit;
    return launch_gemm(g, static_cast<cudaStream_t>(cuda_stream)) == cudaSuccess ? PSATD_OK : PSATD_ERR_CUDA;
}

psatd_status psatd_gemm_bf16_tma(int M, int N, int K, const void* A, const void* B, float* C, void* cuda_stream) {
    if (!A || !B || !C) return PSATD_ERR_ARG;
    const cudaError_t e = launch_gemm_tma(A, B, C, M, N, K, static_cast<cudaStream_t>(cuda_stream));
    if (e == cudaErrorInvalidValue) return PSATD_ERR_ARG;
    return e == cudaSuccess ? PSATD_OK : PSATD_ERR_CUDA;
}

psatd_status psatd_gemm_synchronize(void* cuda_stream) {
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream)) != cudaSuccess) return PSATD_ERR_CUDA;
    return gemm_take_error() ? PSATD_ERR_TIMEOUT : PSATD_OK;
}

psatd_status psatd_fno_synchronize(psatd_fno* f) {
    if (!f) return PSATD_ERR_ARG;
    FCK(cudaStreamSynchronize(f->stream));
    if (gemm_take_error()) return fno_fail(f, PSATD_ERR_TIMEOUT, "a bounded wait in the tensor-core GEMM expired");
    return PSATD_OK;
}

}  // extern "C"
