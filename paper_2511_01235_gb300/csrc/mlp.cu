// A small fully connected network that picks the schedule of an update:
// how many push/relabel cycles per vertex (Alg. 2's KERNEL_CYCLES), how many
// discharge rounds between two global relabels, and whether to repair the
// current flow incrementally (Alg. 5) or re-solve from zero flow (Alg. 1).
// Sec. 6.1 notes that the cycle count trades BFS work against flow sent the
// wrong way, and Sec. 6.2 that the batch size beyond which the static solve
// wins depends on the graph: the network learns both from the solver's own
// timings.  It only steers work; the flow stays exact.
//
// Network: x (n_in) -> relu(W1 x + b1) (H) -> relu(W2 h1 + b2) (H) -> W3 h2 + b3
// (n_out), fp32.  Parameters are one flat vector [W1 | b1 | W2 | b2 | W3 | b3],
// row-major weights (W1 is H x n_in).  Training minimises the masked mean
// squared error between the outputs and target log-latencies with Adam.
// Everything runs in the kernels below: one CTA per sample row for the
// forward and backward passes (activations in shared memory), gradient sums
// by atomics, and an elementwise Adam step.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/maxflow.h"

void mf_note_launches(int kernels);   // the library's launch counter (api.cu)

#define MLP_MAX_IN 64
#define MLP_MAX_H 256
#define MLP_MAX_OUT 64

struct maxflow_mlp {
    int n_in = 0, H = 0, n_out = 0;
    int64_t np = 0;                 // parameter count
    float *p = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;
    float *x = nullptr, *t = nullptr, *mask = nullptr, *y = nullptr, *loss = nullptr;
    int rows_cap = 0;
    double mask_count = 0;          // sum of the mask of the rows last uploaded
    long long step = 0;
    cudaStream_t stream = nullptr;
};

namespace {

struct Layout {
    int n_in, H, n_out;
    __host__ __device__ int w1() const { return 0; }
    __host__ __device__ int b1() const { return H * n_in; }
    __host__ __device__ int w2() const { return b1() + H; }
    __host__ __device__ int b2() const { return w2() + H * H; }
    __host__ __device__ int w3() const { return b2() + H; }
    __host__ __device__ int b3() const { return w3() + n_out * H; }
    __host__ __device__ int total() const { return b3() + n_out; }
};

// Forward pass of one row per CTA (blockDim.x >= max(H, n_out)).
// With t != nullptr it also runs the backward pass of the masked squared
// error and adds this row's gradient into g and its loss into *loss.
__global__ void k_mlp_fwd_bwd(Layout L, const float *__restrict__ p, const float *__restrict__ x,
                              const float *__restrict__ t, const float *__restrict__ mask, float inv_count,
                              float *__restrict__ y, float *__restrict__ g, float *__restrict__ loss)
{
    __shared__ float xs[MLP_MAX_IN], h1[MLP_MAX_H], h2[MLP_MAX_H], d2[MLP_MAX_H], d1[MLP_MAX_H], dy[MLP_MAX_OUT];
    const int r = blockIdx.x, j = threadIdx.x;
    const float *xr = x + (size_t)r * L.n_in;
    if (j < L.n_in) xs[j] = xr[j];
    __syncthreads();
    if (j < L.H) {
        float a = p[L.b1() + j];
        for (int i = 0; i < L.n_in; ++i) a += p[L.w1() + j * L.n_in + i] * xs[i];
        h1[j] = a > 0.f ? a : 0.f;
    }
    __syncthreads();
    if (j < L.H) {
        float a = p[L.b2() + j];
        for (int k = 0; k < L.H; ++k) a += p[L.w2() + j * L.H + k] * h1[k];
        h2[j] = a > 0.f ? a : 0.f;
    }
    __syncthreads();
    if (j < L.n_out) {
        float a = p[L.b3() + j];
        for (int k = 0; k < L.H; ++k) a += p[L.w3() + j * L.H + k] * h2[k];
        y[(size_t)r * L.n_out + j] = a;
        if (t) {
            const float m = mask[(size_t)r * L.n_out + j];
            const float diff = a - t[(size_t)r * L.n_out + j];
            dy[j] = 2.f * m * diff * inv_count;
            if (m != 0.f) atomicAdd(loss, m * diff * diff * inv_count);
        }
    }
    if (!t) return;
    __syncthreads();
    // output layer
    if (j < L.n_out) {
        atomicAdd(g + L.b3() + j, dy[j]);
        for (int k = 0; k < L.H; ++k) atomicAdd(g + L.w3() + j * L.H + k, dy[j] * h2[k]);
    }
    if (j < L.H) {
        float a = 0.f;
        for (int o = 0; o < L.n_out; ++o) a += p[L.w3() + o * L.H + j] * dy[o];
        d2[j] = h2[j] > 0.f ? a : 0.f;
    }
    __syncthreads();
    if (j < L.H) {
        atomicAdd(g + L.b2() + j, d2[j]);
        for (int k = 0; k < L.H; ++k) atomicAdd(g + L.w2() + j * L.H + k, d2[j] * h1[k]);
        float a = 0.f;
        for (int o = 0; o < L.H; ++o) a += p[L.w2() + o * L.H + j] * d2[o];
        d1[j] = h1[j] > 0.f ? a : 0.f;
    }
    __syncthreads();
    if (j < L.H) {
        atomicAdd(g + L.b1() + j, d1[j]);
        for (int i = 0; i < L.n_in; ++i) atomicAdd(g + L.w1() + j * L.n_in + i, d1[j] * xs[i]);
    }
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// p -= lr * m_hat / (sqrt(v_hat) + eps).
__global__ void k_adam(float *p, const float *g, float *m1, float *m2, int64_t np, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float a = b1 * m1[i] + (1.f - b1) * gi;
        const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
        m1[i] = a;
        m2[i] = b;
        p[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
    }
}

int ok(cudaError_t e) { return e == cudaSuccess ? MAXFLOW_OK : MAXFLOW_ERR_CUDA; }

int ensure_rows(maxflow_mlp *m, int rows)
{
    if (rows <= m->rows_cap) return MAXFLOW_OK;
    cudaFree(m->x);
    cudaFree(m->t);
    cudaFree(m->mask);
    cudaFree(m->y);
    m->x = m->t = m->mask = m->y = nullptr;
    size_t ri = (size_t)rows * m->n_in, ro = (size_t)rows * m->n_out;
    if (cudaMalloc(&m->x, ri * sizeof(float)) != cudaSuccess || cudaMalloc(&m->t, ro * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&m->mask, ro * sizeof(float)) != cudaSuccess || cudaMalloc(&m->y, ro * sizeof(float)) != cudaSuccess)
        return MAXFLOW_ERR_OOM;
    m->rows_cap = rows;
    return MAXFLOW_OK;
}

int threads_for(const maxflow_mlp *m)
{
    int need = m->H > m->n_out ? m->H : m->n_out;
    if (m->n_in > need) need = m->n_in;
    return ((need + 31) / 32) * 32;
}

}  // namespace

extern "C" {

int maxflow_mlp_create(maxflow_mlp **out, int32_t n_in, int32_t n_hidden, int32_t n_out, uint64_t seed, void *stream)
{
    if (!out) return MAXFLOW_ERR_INVALID;
    *out = nullptr;
    if (n_in < 1 || n_in > MLP_MAX_IN || n_hidden < 1 || n_hidden > MLP_MAX_H || n_out < 1 || n_out > MLP_MAX_OUT)
        return MAXFLOW_ERR_INVALID;
    maxflow_mlp *m = new (std::nothrow) maxflow_mlp();
    if (!m) return MAXFLOW_ERR_OOM;
    m->n_in = n_in;
    m->H = n_hidden;
    m->n_out = n_out;
    m->stream = (cudaStream_t)stream;
    Layout L{n_in, n_hidden, n_out};
    m->np = L.total();
    int rc = MAXFLOW_OK;
    size_t b = sizeof(float) * (size_t)m->np;
    if (cudaMalloc(&m->p, b) != cudaSuccess || cudaMalloc(&m->g, b) != cudaSuccess ||
        cudaMalloc(&m->m1, b) != cudaSuccess || cudaMalloc(&m->m2, b) != cudaSuccess ||
        cudaMalloc(&m->loss, sizeof(float)) != cudaSuccess)
        rc = MAXFLOW_ERR_OOM;
    if (rc == MAXFLOW_OK) {
        // He-uniform weights from a 64-bit linear congruential generator, zero biases
        std::vector<float> h((size_t)m->np, 0.f);
        uint64_t st = seed * 6364136223846793005ull + 1442695040888963407ull;
        auto uni = [&]() {
            st = st * 6364136223846793005ull + 1442695040888963407ull;
            return (float)((st >> 11) * (1.0 / 9007199254740992.0)) * 2.f - 1.f;
        };
        const float s1 = std::sqrt(6.f / (float)n_in), s2 = std::sqrt(6.f / (float)n_hidden);
        for (int i = 0; i < n_hidden * n_in; ++i) h[(size_t)L.w1() + i] = s1 * uni();
        for (int i = 0; i < n_hidden * n_hidden; ++i) h[(size_t)L.w2() + i] = s2 * uni();
        for (int i = 0; i < n_out * n_hidden; ++i) h[(size_t)L.w3() + i] = s2 * uni();
        rc = ok(cudaMemcpy(m->p, h.data(), b, cudaMemcpyHostToDevice));
        if (rc == MAXFLOW_OK) rc = ok(cudaMemset(m->m1, 0, b));
        if (rc == MAXFLOW_OK) rc = ok(cudaMemset(m->m2, 0, b));
    }
    if (rc != MAXFLOW_OK) {
        maxflow_mlp_destroy(m);
        return rc;
    }
    *out = m;
    return MAXFLOW_OK;
}

void maxflow_mlp_destroy(maxflow_mlp *m)
{
    if (!m) return;
    cudaFree(m->p);
    cudaFree(m->g);
    cudaFree(m->m1);
    cudaFree(m->m2);
    cudaFree(m->x);
    cudaFree(m->t);
    cudaFree(m->mask);
    cudaFree(m->y);
    cudaFree(m->loss);
    delete m;
}

int maxflow_mlp_shape(maxflow_mlp *m, int32_t *n_in, int32_t *n_hidden, int32_t *n_out, int64_t *n_params)
{
    if (!m) return MAXFLOW_ERR_INVALID;
    if (n_in) *n_in = m->n_in;
    if (n_hidden) *n_hidden = m->H;
    if (n_out) *n_out = m->n_out;
    if (n_params) *n_params = m->np;
    return MAXFLOW_OK;
}

int maxflow_mlp_get_params(maxflow_mlp *m, float *host, int64_t count)
{
    if (!m || !host || count != m->np) return MAXFLOW_ERR_INVALID;
    return ok(cudaMemcpy(host, m->p, sizeof(float) * (size_t)count, cudaMemcpyDeviceToHost));
}

int maxflow_mlp_set_params(maxflow_mlp *m, const float *host, int64_t count)
{
    if (!m || !host || count != m->np) return MAXFLOW_ERR_INVALID;
    m->step = 0;
    size_t b = sizeof(float) * (size_t)count;
    int rc = ok(cudaMemcpy(m->p, host, b, cudaMemcpyHostToDevice));
    if (rc == MAXFLOW_OK) rc = ok(cudaMemset(m->m1, 0, b));
    if (rc == MAXFLOW_OK) rc = ok(cudaMemset(m->m2, 0, b));
    return rc;
}

int maxflow_mlp_forward(maxflow_mlp *m, const float *x, int32_t rows, float *y)
{
    if (!m || !x || !y || rows < 1) return MAXFLOW_ERR_INVALID;
    int rc = ensure_rows(m, rows);
    if (rc != MAXFLOW_OK) return rc;
    rc = ok(cudaMemcpyAsync(m->x, x, sizeof(float) * (size_t)rows * m->n_in, cudaMemcpyHostToDevice, m->stream));
    Layout L{m->n_in, m->H, m->n_out};
    if (rc == MAXFLOW_OK) {
        k_mlp_fwd_bwd<<<rows, threads_for(m), 0, m->stream>>>(L, m->p, m->x, nullptr, nullptr, 0.f, m->y, nullptr,
                                                              nullptr);
        rc = ok(cudaGetLastError());
        if (rc == MAXFLOW_OK) mf_note_launches(1);
    }
    if (rc == MAXFLOW_OK)
        rc = ok(cudaMemcpyAsync(y, m->y, sizeof(float) * (size_t)rows * m->n_out, cudaMemcpyDeviceToHost, m->stream));
    if (rc == MAXFLOW_OK) rc = ok(cudaStreamSynchronize(m->stream));
    return rc;
}

// Device-side forward for the scheduler (x, y device pointers, no sync).
int mlp_forward_device(maxflow_mlp *m, const float *x_dev, int32_t rows, float *y_dev, cudaStream_t st)
{
    Layout L{m->n_in, m->H, m->n_out};
    k_mlp_fwd_bwd<<<rows, threads_for(m), 0, st>>>(L, m->p, x_dev, nullptr, nullptr, 0.f, y_dev, nullptr, nullptr);
    int rc = ok(cudaGetLastError());
    if (rc == MAXFLOW_OK) mf_note_launches(1);
    return rc;
}

int mlp_n_out(const maxflow_mlp *m) { return m->n_out; }
int mlp_n_in(const maxflow_mlp *m) { return m->n_in; }

static int grad_pass(maxflow_mlp *m, int32_t rows, float *loss_host)
{
    Layout L{m->n_in, m->H, m->n_out};
    const double cnt = m->mask_count;
    if (cnt <= 0) return MAXFLOW_ERR_INVALID;
    int rc = ok(cudaMemsetAsync(m->g, 0, sizeof(float) * (size_t)m->np, m->stream));
    if (rc == MAXFLOW_OK) rc = ok(cudaMemsetAsync(m->loss, 0, sizeof(float), m->stream));
    if (rc == MAXFLOW_OK) {
        k_mlp_fwd_bwd<<<rows, threads_for(m), 0, m->stream>>>(L, m->p, m->x, m->t, m->mask, (float)(1.0 / cnt),
                                                              m->y, m->g, m->loss);
        rc = ok(cudaGetLastError());
        if (rc == MAXFLOW_OK) mf_note_launches(1);
    }
    if (rc == MAXFLOW_OK && loss_host) {
        rc = ok(cudaMemcpyAsync(loss_host, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
        if (rc == MAXFLOW_OK) rc = ok(cudaStreamSynchronize(m->stream));
    }
    return rc;
}

static int upload_rows(maxflow_mlp *m, const float *x, const float *t, const float *mask, int32_t rows)
{
    double cnt = 0;
    for (size_t i = 0; i < (size_t)rows * m->n_out; ++i) {
        if (!(mask[i] >= 0.f)) return MAXFLOW_ERR_INVALID;
        cnt += mask[i];
    }
    m->mask_count = cnt;
    int rc = ensure_rows(m, rows);
    if (rc != MAXFLOW_OK) return rc;
    rc = ok(cudaMemcpyAsync(m->x, x, sizeof(float) * (size_t)rows * m->n_in, cudaMemcpyHostToDevice, m->stream));
    if (rc == MAXFLOW_OK)
        rc = ok(cudaMemcpyAsync(m->t, t, sizeof(float) * (size_t)rows * m->n_out, cudaMemcpyHostToDevice, m->stream));
    if (rc == MAXFLOW_OK)
        rc = ok(cudaMemcpyAsync(m->mask, mask, sizeof(float) * (size_t)rows * m->n_out, cudaMemcpyHostToDevice,
                                m->stream));
    return rc;
}

int maxflow_mlp_grad(maxflow_mlp *m, const float *x, const float *t, const float *mask, int32_t rows, float *grad,
                     float *loss)
{
    if (!m || !x || !t || !mask || rows < 1 || !grad) return MAXFLOW_ERR_INVALID;
    int rc = upload_rows(m, x, t, mask, rows);
    if (rc == MAXFLOW_OK) rc = grad_pass(m, rows, loss);
    if (rc == MAXFLOW_OK)
        rc = ok(cudaMemcpyAsync(grad, m->g, sizeof(float) * (size_t)m->np, cudaMemcpyDeviceToHost, m->stream));
    if (rc == MAXFLOW_OK) rc = ok(cudaStreamSynchronize(m->stream));
    return rc;
}

int maxflow_mlp_train(maxflow_mlp *m, const float *x, const float *t, const float *mask, int32_t rows, int32_t steps,
                      float lr, float *loss_last)
{
    if (!m || !x || !t || !mask || rows < 1 || steps < 1 || !(lr > 0.f)) return MAXFLOW_ERR_INVALID;
    int rc = upload_rows(m, x, t, mask, rows);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int s = 0; s < steps && rc == MAXFLOW_OK; ++s) {
        rc = grad_pass(m, rows, (s == steps - 1) ? loss_last : nullptr);
        if (rc != MAXFLOW_OK) break;
        m->step += 1;
        const float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
        int g = (int)((m->np + 255) / 256);
        k_adam<<<g, 256, 0, m->stream>>>(m->p, m->g, m->m1, m->m2, m->np, lr, b1, b2, eps, c1, c2);
        rc = ok(cudaGetLastError());
        if (rc == MAXFLOW_OK) mf_note_launches(1);
    }
    if (rc == MAXFLOW_OK) rc = ok(cudaStreamSynchronize(m->stream));
    return rc;
}

}  // extern "C"
