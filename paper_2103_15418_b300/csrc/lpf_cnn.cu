// C ABI of the parameter-inference network on the dynamic-spectrum batch
// (include/lpf.h, lpf_cnn_*); the kernels are in lpf_cnn.cuh.
#include "../../include/lpf.h"
#include "lpf_cnn.cuh"

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

struct lpf_cnn {
    int dev = 0;
    int F = 0, Tw = 0, max_batch = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    float* w1 = nullptr;              // conv1 [16][9] FP32
    float* b1 = nullptr;              // [16]
    __nv_bfloat16* w2 = nullptr;      // conv2 [32][9 * 16] BF16, k = tap * 16 + c
    float* b2 = nullptr;
    __nv_bfloat16* w3 = nullptr;      // conv3 [64][9 * 32] BF16
    float* b3 = nullptr;
    float* hw = nullptr;              // head [5][64]
    float* hb = nullptr;              // [5]
    __nv_bfloat16* act1 = nullptr;    // [max_batch][F/2][Tw/2][16]
    __nv_bfloat16* act2 = nullptr;    // [max_batch][F/4][Tw/4][32]
    unsigned* err = nullptr;          // bit 0: an MMA completion wait ran out
    int n_sm = 0;
    bool fused = false;               // 32 x 64 spectra: the one-kernel network
};

namespace {

using namespace lpf::cnn;

void cnn_free(lpf_cnn* c) {
    if (!c) return;
    cudaSetDevice(c->dev);
    if (c->st) cudaStreamSynchronize(c->st);
    void* p[] = {c->w1, c->b1, c->w2, c->b2, c->w3, c->b3, c->hw, c->hb, c->act1, c->act2, c->err};
    for (void* q : p)
        if (q) cudaFree(q);
    if (c->own_stream && c->st) cudaStreamDestroy(c->st);
}

template <typename T>
int upload(T** dst, const T* src, size_t n) {
    if (cudaMalloc((void**)dst, std::max<size_t>(n * sizeof(T), 16)) != cudaSuccess) {
        cudaGetLastError();
        *dst = nullptr;
        return LPF_E_OOM;
    }
    if (src && cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) return LPF_E_CUDA;
    return LPF_OK;
}

// OIHW FP32 weights [cout][cin][3][3] -> BF16 [cout][9 cin], k = (ky 3 + kx) cin + c
std::vector<__nv_bfloat16> gemm_weights(const float* w, int cout, int cin) {
    std::vector<__nv_bfloat16> o((size_t)cout * 9 * cin);
    for (int n = 0; n < cout; ++n)
        for (int c = 0; c < cin; ++c)
            for (int tap = 0; tap < 9; ++tap)
                o[(size_t)n * 9 * cin + tap * cin + c] = __float2bfloat16_rn(w[((size_t)n * cin + c) * 9 + tap]);
    return o;
}

bool pow2_le(int v, int cap) { return v >= 1 && v <= cap && (v & (v - 1)) == 0; }

}  // namespace

extern "C" {

size_t lpf_cnn_param_count(void) {
    return (size_t)kC1 * 9 + kC1 + (size_t)kC2 * kC1 * 9 + kC2 + (size_t)kC3 * kC2 * 9 + kC3 + (size_t)kOut * kC3 + kOut;
}

int lpf_cnn_open(lpf_cnn** out, int F, int Tw, const float* params, size_t n_params, int max_batch,
                 void* cuda_stream) {
    if (!out) return LPF_E_ARG;
    *out = nullptr;
    if (!params || n_params != lpf_cnn_param_count() || max_batch < 1) return LPF_E_ARG;
    // two 2x2 means, and a spectrum's pixels at conv3 a power of two <= 128
    if (F < 4 || Tw < 4 || F % 4 || Tw % 4 || !pow2_le((F / 4) * (Tw / 4), kRows)) return LPF_E_ARG;
    if ((int64_t)max_batch * F * Tw > ((int64_t)1 << 31)) return LPF_E_ARG;
    lpf_cnn* c = new (std::nothrow) lpf_cnn();
    if (!c) return LPF_E_OOM;
    c->F = F; c->Tw = Tw; c->max_batch = max_batch;
    int ndev = 0;
    if (cudaGetDevice(&c->dev) != cudaSuccess || cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        delete c;
        return LPF_E_CUDA;
    }
    int rc = LPF_OK;
    if (cuda_stream) {
        c->st = (cudaStream_t)cuda_stream;
    } else if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess) {
        rc = LPF_E_CUDA;
    } else {
        c->own_stream = true;
    }
    const float* p = params;
    const float* w1 = p; p += kC1 * 9;
    const float* b1 = p; p += kC1;
    const float* w2 = p; p += kC2 * kC1 * 9;
    const float* b2 = p; p += kC2;
    const float* w3 = p; p += kC3 * kC2 * 9;
    const float* b3 = p; p += kC3;
    const float* hw = p; p += kOut * kC3;
    const float* hb = p;
    const std::vector<__nv_bfloat16> g2 = gemm_weights(w2, kC2, kC1), g3 = gemm_weights(w3, kC3, kC2);
    if (rc == LPF_OK) rc = upload(&c->w1, w1, (size_t)kC1 * 9);
    if (rc == LPF_OK) rc = upload(&c->b1, b1, kC1);
    if (rc == LPF_OK) rc = upload(&c->w2, g2.data(), g2.size());
    if (rc == LPF_OK) rc = upload(&c->b2, b2, kC2);
    if (rc == LPF_OK) rc = upload(&c->w3, g3.data(), g3.size());
    if (rc == LPF_OK) rc = upload(&c->b3, b3, kC3);
    if (rc == LPF_OK) rc = upload(&c->hw, hw, (size_t)kOut * kC3);
    if (rc == LPF_OK) rc = upload(&c->hb, hb, kOut);
    if (rc == LPF_OK) rc = upload<__nv_bfloat16>(&c->act1, nullptr, (size_t)max_batch * (F / 2) * (Tw / 2) * kC1);
    if (rc == LPF_OK) rc = upload<__nv_bfloat16>(&c->act2, nullptr, (size_t)max_batch * (F / 4) * (Tw / 4) * kC2);
    if (rc == LPF_OK) rc = upload<unsigned>(&c->err, nullptr, 1);
    if (rc == LPF_OK && cudaMemset(c->err, 0, sizeof(unsigned)) != cudaSuccess) rc = LPF_E_CUDA;
    if (rc == LPF_OK && cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->dev) != cudaSuccess)
        rc = LPF_E_CUDA;
    c->fused = F == fused::H0 && Tw == fused::W0;
    if (rc == LPF_OK && c->fused &&
        cudaFuncSetAttribute(k_cnn_fused_32x64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fused::SMEM) !=
            cudaSuccess)
        rc = LPF_E_CUDA;
    if (rc == LPF_OK &&
        (cudaFuncSetAttribute(k_cnn_conv_tc<kC1, kC2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)conv_tc_smem_bytes<kC1, kC2>()) != cudaSuccess ||
         cudaFuncSetAttribute(k_cnn_conv_tc<kC2, kC3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)conv_tc_smem_bytes<kC2, kC3>()) != cudaSuccess))
        rc = LPF_E_CUDA;
    if (rc != LPF_OK) {
        cnn_free(c);
        delete c;
        return rc;
    }
    *out = c;
    return LPF_OK;
}

int lpf_cnn_forward(lpf_cnn* c, const float* x_dev, int n, float* out_dev) {
    if (!c || n < 0 || n > c->max_batch || (n > 0 && (!x_dev || !out_dev))) return LPF_E_ARG;
    if (n == 0) return LPF_OK;
    if (cudaSetDevice(c->dev) != cudaSuccess) return LPF_E_CUDA;
    cudaGetLastError();
    const int F = c->F, Tw = c->Tw;
    if (c->fused) {
        if (reinterpret_cast<uintptr_t>(x_dev) & 15u) return LPF_E_ARG;   // 16-byte copies of each spectrum
        const int grid = std::min(n, 2 * c->n_sm);
        k_cnn_fused_32x64<<<grid, kRows, fused::SMEM, c->st>>>(x_dev, n, c->w1, c->b1, c->w2, c->b2, c->w3, c->b3,
                                                              c->hw, c->hb, out_dev, c->err);
        return cudaGetLastError() == cudaSuccess ? LPF_OK : LPF_E_CUDA;
    }
    const int64_t win1 = (int64_t)n * (F / 2) * (Tw / 2);
    const int g1 = (int)std::min<int64_t>((win1 + 255) / 256, 148 * 16);
    k_cnn_conv1<<<g1, 256, 0, c->st>>>(x_dev, n, F, Tw, c->w1, c->b1, c->act1);
    const int64_t m2 = (int64_t)n * (F / 2) * (Tw / 2), m3 = (int64_t)n * (F / 4) * (Tw / 4);
    k_cnn_conv_tc<kC1, kC2, false><<<(unsigned)((m2 + kRows - 1) / kRows), kRows, conv_tc_smem_bytes<kC1, kC2>(),
                                     c->st>>>(c->act1, n, F / 2, Tw / 2, c->w2, c->b2, c->act2, nullptr, nullptr,
                                              nullptr, c->err);
    k_cnn_conv_tc<kC2, kC3, true><<<(unsigned)((m3 + kRows - 1) / kRows), kRows, conv_tc_smem_bytes<kC2, kC3>(),
                                    c->st>>>(c->act2, n, F / 4, Tw / 4, c->w3, c->b3, nullptr, c->hw, c->hb, out_dev,
                                             c->err);
    return cudaGetLastError() == cudaSuccess ? LPF_OK : LPF_E_CUDA;
}

int lpf_cnn_sync(lpf_cnn* c) {
    if (!c) return LPF_E_ARG;
    if (cudaSetDevice(c->dev) != cudaSuccess || cudaStreamSynchronize(c->st) != cudaSuccess) return LPF_E_CUDA;
    unsigned e = 0;
    if (cudaMemcpy(&e, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return LPF_E_CUDA;
    return e ? LPF_E_TIMEOUT : LPF_OK;
}

int lpf_cnn_close(lpf_cnn* c) {
    if (!c) return LPF_OK;
    cnn_free(c);
    delete c;
    return LPF_OK;
}

}  // extern "C"
