// mlp.cu -- the small fp32 multilayer perceptron that predicts a code's termination
// level and distance from mdist_features (used only to size and order work): hand-
// written forward, backward (MSE loss) and Adam kernels, and its C-ABI.
//
// Layout: layer l maps in_l -> out_l with W_l (in_l x out_l, row-major) and b_l;
// hidden layers use ReLU, the last layer is linear.  Parameters are stored layer
// after layer: W_0, b_0, W_1, b_1, ...
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

namespace mdist {
namespace {

__host__ __device__ inline unsigned long long splitmix64(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// minibatch rows drawn with replacement: row b of step s is hash(seed, s * B + b) mod N
__global__ void mlp_gather(const float *X, const float *T, float *Xb, float *Tb, int N, int B, int F, int O,
                           unsigned long long seed, int step) {
    const int b = blockIdx.x;
    if (b >= B) return;
    const int idx = (int)(splitmix64(seed ^ splitmix64((unsigned long long)step * B + b)) % (unsigned long long)N);
    for (int i = threadIdx.x; i < F; i += blockDim.x) Xb[(size_t)b * F + i] = X[(size_t)idx * F + i];
    for (int i = threadIdx.x; i < O; i += blockDim.x) Tb[(size_t)b * O + i] = T[(size_t)idx * O + i];
}

// Y[b][o] = bias[o] + sum_i X[b][i] W[i][o], then ReLU if relu
__global__ void mlp_linear_fwd(const float *X, const float *Wt, const float *bias, float *Y, int B, int I, int O,
                               int relu) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * O) return;
    const int b = t / O, o = t - b * O;
    float acc = bias[o];
    for (int i = 0; i < I; ++i) acc = fmaf(X[(size_t)b * I + i], Wt[(size_t)i * O + o], acc);
    Y[t] = relu ? fmaxf(acc, 0.f) : acc;
}

// loss = mean over B*O of (Y - T)^2; dY = 2 (Y - T) / (B * O)
__global__ void mlp_mse(const float *Y, const float *T, float *dY, float *loss, int n) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    float e = 0.f;
    if (t < n) {
        const float d = Y[t] - T[t];
        dY[t] = 2.f * d / (float)n;
        e = d * d / (float)n;
    }
    for (int off = 16; off > 0; off >>= 1) e += __shfl_down_sync(0xffffffffu, e, off);
    if ((threadIdx.x & 31) == 0 && e != 0.f) atomicAdd(loss, e);
}

// dW[i][o] = sum_b X[b][i] dY[b][o]; the extra row i = I is the bias gradient
__global__ void mlp_linear_bwd_param(const float *X, const float *dY, float *dW, float *db, int B, int I, int O) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (I + 1) * O) return;
    const int i = t / O, o = t - i * O;
    float acc = 0.f;
    if (i < I) {
        for (int b = 0; b < B; ++b) acc = fmaf(X[(size_t)b * I + i], dY[(size_t)b * O + o], acc);
        dW[t] = acc;
    } else {
        for (int b = 0; b < B; ++b) acc += dY[(size_t)b * O + o];
        db[o] = acc;
    }
}

// dX[b][i] = (sum_o dY[b][o] W[i][o]) * [X[b][i] > 0]  (X = ReLU output of the layer below)
__global__ void mlp_linear_bwd_data(const float *dY, const float *Wt, const float *X, float *dX, int B, int I, int O) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * I) return;
    const int b = t / I, i = t - b * I;
    float acc = 0.f;
    for (int o = 0; o < O; ++o) acc = fmaf(dY[(size_t)b * O + o], Wt[(size_t)i * O + o], acc);
    dX[t] = X[t] > 0.f ? acc : 0.f;
}

__global__ void mlp_adam(float *P, const float *Gr, float *M, float *V, int n, float lr, float b1, float b2, float eps,
                         float c1, float c2) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float g = Gr[t];
    const float m = b1 * M[t] + (1.f - b1) * g;
    const float v = b2 * V[t] + (1.f - b2) * g * g;
    M[t] = m;
    V[t] = v;
    P[t] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

}  // namespace
}  // namespace mdist

using namespace mdist;

struct mdist_mlp {
    int F = 0, H = 0, layers = 0, O = 0;    // layers = number of linear layers
    std::vector<int> in, out;               // per layer
    std::vector<size_t> woff, boff;         // parameter offsets
    size_t nparams = 0;
    cudaStream_t stream = nullptr;
    float *P = nullptr, *Gr = nullptr, *M = nullptr, *V = nullptr;
    float *loss = nullptr;
    int adam_t = 0;
    // work buffers for a batch of up to cap rows
    int cap = 0;
    std::vector<float *> act;               // act[0] = input, act[l + 1] = layer l output
    std::vector<float *> grad;              // grad[l] = dLoss / d act[l]
    float *Tb = nullptr;
    std::vector<void *> allocs;
};

namespace {

void *mlp_alloc(mdist_mlp *m, size_t bytes) {
    void *p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 4) != cudaSuccess) return nullptr;
    m->allocs.push_back(p);
    return p;
}

void mlp_release(void *p) { cudaFree(p); }

int ensure_batch(mdist_mlp *m, int B) {
    if (B <= m->cap) return MDIST_OK;
    for (float *p : m->act) {
        for (auto it = m->allocs.begin(); it != m->allocs.end(); ++it)
            if (*it == p) { m->allocs.erase(it); break; }
        mlp_release(p);
    }
    for (float *p : m->grad) {
        for (auto it = m->allocs.begin(); it != m->allocs.end(); ++it)
            if (*it == p) { m->allocs.erase(it); break; }
        mlp_release(p);
    }
    if (m->Tb) {
        for (auto it = m->allocs.begin(); it != m->allocs.end(); ++it)
            if (*it == m->Tb) { m->allocs.erase(it); break; }
        mlp_release(m->Tb);
    }
    m->act.assign((size_t)m->layers + 1, nullptr);
    m->grad.assign((size_t)m->layers + 1, nullptr);
    for (int l = 0; l <= m->layers; ++l) {
        const int width = l == 0 ? m->F : m->out[(size_t)l - 1];
        m->act[(size_t)l] = (float *)mlp_alloc(m, sizeof(float) * (size_t)B * width);
        m->grad[(size_t)l] = (float *)mlp_alloc(m, sizeof(float) * (size_t)B * width);
        if (!m->act[(size_t)l] || !m->grad[(size_t)l]) return MDIST_ENOMEM;
    }
    m->Tb = (float *)mlp_alloc(m, sizeof(float) * (size_t)B * m->O);
    if (!m->Tb) return MDIST_ENOMEM;
    m->cap = B;
    return MDIST_OK;
}

inline int nblk(long long n) { return (int)((n + 255) / 256); }

void forward(mdist_mlp *m, int B) {
    for (int l = 0; l < m->layers; ++l) {
        const int I = m->in[(size_t)l], O = m->out[(size_t)l];
        mlp_linear_fwd<<<nblk((long long)B * O), 256, 0, m->stream>>>(m->act[(size_t)l], m->P + m->woff[(size_t)l],
                                                                     m->P + m->boff[(size_t)l], m->act[(size_t)l + 1], B,
                                                                     I, O, l + 1 < m->layers ? 1 : 0);
    }
}

// loss and gradients of the batch already in act[0] / Tb; gradients land in Gr
void backward(mdist_mlp *m, int B) {
    const int L = m->layers;
    cudaMemsetAsync(m->loss, 0, sizeof(float), m->stream);
    mlp_mse<<<nblk((long long)B * m->O), 256, 0, m->stream>>>(m->act[(size_t)L], m->Tb, m->grad[(size_t)L], m->loss,
                                                             B * m->O);
    for (int l = L - 1; l >= 0; --l) {
        const int I = m->in[(size_t)l], O = m->out[(size_t)l];
        mlp_linear_bwd_param<<<nblk((long long)(I + 1) * O), 256, 0, m->stream>>>(
            m->act[(size_t)l], m->grad[(size_t)l + 1], m->Gr + m->woff[(size_t)l], m->Gr + m->boff[(size_t)l], B, I, O);
        if (l > 0)
            mlp_linear_bwd_data<<<nblk((long long)B * I), 256, 0, m->stream>>>(
                m->grad[(size_t)l + 1], m->P + m->woff[(size_t)l], m->act[(size_t)l], m->grad[(size_t)l], B, I, O);
    }
}

}  // namespace

extern "C" {

int mdist_mlp_create(int in_features, int hidden, int hidden_layers, int outputs, uint64_t seed, void *cuda_stream,
                     mdist_mlp **out) {
    if (!out || in_features < 1 || hidden < 1 || hidden_layers < 0 || outputs < 1 || in_features > 4096 ||
        hidden > 4096 || hidden_layers > 16 || outputs > 4096)
        return MDIST_EINVAL;
    *out = nullptr;
    mdist_mlp *m = new (std::nothrow) mdist_mlp();
    if (!m) return MDIST_ENOMEM;
    m->F = in_features;
    m->H = hidden;
    m->O = outputs;
    m->layers = hidden_layers + 1;
    m->stream = (cudaStream_t)cuda_stream;
    size_t off = 0;
    for (int l = 0; l < m->layers; ++l) {
        const int I = l == 0 ? in_features : hidden;
        const int O = l + 1 == m->layers ? outputs : hidden;
        m->in.push_back(I);
        m->out.push_back(O);
        m->woff.push_back(off);
        off += (size_t)I * O;
        m->boff.push_back(off);
        off += (size_t)O;
    }
    m->nparams = off;
    // He-uniform weights from SplitMix64, zero biases
    std::vector<float> h(m->nparams, 0.f);
    unsigned long long s = seed;
    for (int l = 0; l < m->layers; ++l) {
        const float a = std::sqrt(6.0f / (float)m->in[(size_t)l]);
        for (size_t i = 0; i < (size_t)m->in[(size_t)l] * m->out[(size_t)l]; ++i) {
            s += 0x9E3779B97F4A7C15ull;
            const double u = (double)(splitmix64(s) >> 11) * (1.0 / 9007199254740992.0);
            h[m->woff[(size_t)l] + i] = (float)((2.0 * u - 1.0) * a);
        }
    }
    m->P = (float *)mlp_alloc(m, sizeof(float) * m->nparams);
    m->Gr = (float *)mlp_alloc(m, sizeof(float) * m->nparams);
    m->M = (float *)mlp_alloc(m, sizeof(float) * m->nparams);
    m->V = (float *)mlp_alloc(m, sizeof(float) * m->nparams);
    m->loss = (float *)mlp_alloc(m, sizeof(float));
    if (!m->P || !m->Gr || !m->M || !m->V || !m->loss) {
        for (void *p : m->allocs) mlp_release(p);
        delete m;
        return MDIST_ENOMEM;
    }
    cudaMemcpyAsync(m->P, h.data(), sizeof(float) * m->nparams, cudaMemcpyHostToDevice, m->stream);
    cudaMemsetAsync(m->M, 0, sizeof(float) * m->nparams, m->stream);
    cudaMemsetAsync(m->V, 0, sizeof(float) * m->nparams, m->stream);
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) {
        for (void *p : m->allocs) mlp_release(p);
        delete m;
        return MDIST_ECUDA;
    }
    *out = m;
    return MDIST_OK;
}

int mdist_mlp_num_params(const mdist_mlp *m, int *n) {
    if (!m || !n) return MDIST_EINVAL;
    *n = (int)m->nparams;
    return MDIST_OK;
}

int mdist_mlp_get_params(const mdist_mlp *m, float *p) {
    if (!m || !p) return MDIST_EINVAL;
    if (cudaMemcpyAsync(p, m->P, sizeof(float) * m->nparams, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess)
        return MDIST_ECUDA;
    return MDIST_OK;
}

int mdist_mlp_set_params(mdist_mlp *m, const float *p) {
    if (!m || !p) return MDIST_EINVAL;
    if (cudaMemcpyAsync(m->P, p, sizeof(float) * m->nparams, cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess)
        return MDIST_ECUDA;
    m->adam_t = 0;
    cudaMemsetAsync(m->M, 0, sizeof(float) * m->nparams, m->stream);
    cudaMemsetAsync(m->V, 0, sizeof(float) * m->nparams, m->stream);
    return cudaStreamSynchronize(m->stream) == cudaSuccess ? MDIST_OK : MDIST_ECUDA;
}

int mdist_mlp_forward(mdist_mlp *m, const float *X, int N, float *Y) {
    if (!m || !X || !Y || N < 1) return MDIST_EINVAL;
    int rc = ensure_batch(m, N);
    if (rc != MDIST_OK) return rc;
    cudaMemcpyAsync(m->act[0], X, sizeof(float) * (size_t)N * m->F, cudaMemcpyHostToDevice, m->stream);
    forward(m, N);
    cudaMemcpyAsync(Y, m->act[(size_t)m->layers], sizeof(float) * (size_t)N * m->O, cudaMemcpyDeviceToHost, m->stream);
    return cudaStreamSynchronize(m->stream) == cudaSuccess && cudaGetLastError() == cudaSuccess ? MDIST_OK : MDIST_ECUDA;
}

int mdist_mlp_loss_grad(mdist_mlp *m, const float *X, const float *T, int N, float *loss, float *grad) {
    if (!m || !X || !T || N < 1) return MDIST_EINVAL;
    int rc = ensure_batch(m, N);
    if (rc != MDIST_OK) return rc;
    cudaMemcpyAsync(m->act[0], X, sizeof(float) * (size_t)N * m->F, cudaMemcpyHostToDevice, m->stream);
    cudaMemcpyAsync(m->Tb, T, sizeof(float) * (size_t)N * m->O, cudaMemcpyHostToDevice, m->stream);
    forward(m, N);
    backward(m, N);
    if (loss) cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream);
    if (grad) cudaMemcpyAsync(grad, m->Gr, sizeof(float) * m->nparams, cudaMemcpyDeviceToHost, m->stream);
    return cudaStreamSynchronize(m->stream) == cudaSuccess && cudaGetLastError() == cudaSuccess ? MDIST_OK : MDIST_ECUDA;
}

int mdist_mlp_train(mdist_mlp *m, const float *X, const float *T, int N, int steps, int batch, float lr, uint64_t seed,
                    float *loss_curve) {
    if (!m || !X || !T || N < 1 || steps < 1 || batch < 1 || !(lr > 0.f)) return MDIST_EINVAL;
    int rc = ensure_batch(m, batch);
    if (rc != MDIST_OK) return rc;
    float *dX = nullptr, *dT = nullptr, *curve = nullptr;
    if (cudaMalloc(&dX, sizeof(float) * (size_t)N * m->F) != cudaSuccess ||
        cudaMalloc(&dT, sizeof(float) * (size_t)N * m->O) != cudaSuccess ||
        cudaMalloc(&curve, sizeof(float) * (size_t)steps) != cudaSuccess) {
        cudaFree(dX);
        cudaFree(dT);
        return MDIST_ENOMEM;
    }
    cudaMemcpyAsync(dX, X, sizeof(float) * (size_t)N * m->F, cudaMemcpyHostToDevice, m->stream);
    cudaMemcpyAsync(dT, T, sizeof(float) * (size_t)N * m->O, cudaMemcpyHostToDevice, m->stream);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int s = 0; s < steps; ++s) {
        mlp_gather<<<batch, 64, 0, m->stream>>>(dX, dT, m->act[0], m->Tb, N, batch, m->F, m->O, seed, s);
        forward(m, batch);
        backward(m, batch);
        cudaMemcpyAsync(curve + s, m->loss, sizeof(float), cudaMemcpyDeviceToDevice, m->stream);
        m->adam_t += 1;
        const float c1 = 1.f - std::pow(b1, (float)m->adam_t), c2 = 1.f - std::pow(b2, (float)m->adam_t);
        mlp_adam<<<nblk((long long)m->nparams), 256, 0, m->stream>>>(m->P, m->Gr, m->M, m->V, (int)m->nparams, lr, b1,
                                                                     b2, eps, c1, c2);
    }
    if (loss_curve) cudaMemcpyAsync(loss_curve, curve, sizeof(float) * (size_t)steps, cudaMemcpyDeviceToHost, m->stream);
    rc = cudaStreamSynchronize(m->stream) == cudaSuccess && cudaGetLastError() == cudaSuccess ? MDIST_OK : MDIST_ECUDA;
    cudaFree(dX);
    cudaFree(dT);
    cudaFree(curve);
    return rc;
}

void mdist_mlp_free(mdist_mlp *m) {
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    for (void *p : m->allocs) mlp_release(p);
    delete m;
}

}  // extern "C"
