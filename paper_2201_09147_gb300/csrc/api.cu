// C-ABI layer of libsdfnn: network loading and preparation, argument
// validation, and orchestration of the kernels on the caller's stream.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_fp16.h>

#include "../../include/sdfnn.h"
#include "common.cuh"
#include "internal.h"

using namespace sdfnn;

struct sdf_net {
    int device = 0;
    int precision = SDF_FP32;
    int in_dim = 3, width = 0, n_hidden = 0;
    double lipschitz = 0.0;
    float time = 0.0f;
    float bout = 0.0f;
    float* d_f32 = nullptr;       // folded FP32 parameters
    std::vector<float> h_f32;     // the same, on the host (launch parameters of the width-64 trace)
    uint8_t* d_bf16 = nullptr;    // swizzled 16-bit hidden weights (SDF_BF16 / SDF_FP16)
    size_t off_w0 = 0, off_b0 = 0, off_wt[kMaxHidden] = {}, off_bh[kMaxHidden] = {}, off_wout = 0;
    uint32_t bf16_layer_bytes = 0;
    int rows_pad = 0;
    float q_w[kMaxHidden] = {}, q_g[kMaxHidden + 1] = {}, q_o = 1.0f;  // SDF_FP8 scales
};

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(SDF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

struct DeviceInfo {
    int num_sms = 0;
    int* d_status = nullptr;
    cudaMemPool_t pool = nullptr;  // the library's stream-ordered pool for per-call scratch
};

std::mutex g_dev_mutex;
std::vector<DeviceInfo> g_devices;

// Per-device SM count and status word (allocated once, kept until exit).
// The caller has already made `dev` current.
int device_info(int dev, DeviceInfo* out) {
    std::lock_guard<std::mutex> lock(g_dev_mutex);
    if (static_cast<int>(g_devices.size()) <= dev) g_devices.resize(dev + 1);
    DeviceInfo& d = g_devices[dev];
    if (d.num_sms == 0) {
        // Filled in a local record and published only once complete, so a
        // failed step is retried by the next call instead of leaving a record
        // without its status word or pool.
        DeviceInfo n;
        cudaError_t e = cudaDeviceGetAttribute(&n.num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
        e = cudaMalloc(&n.d_status, sizeof(int));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(status)");
        e = cudaMemset(n.d_status, 0, sizeof(int));
        if (e != cudaSuccess) {
            cudaFree(n.d_status);
            return cuda_fail(e, "cudaMemset(status)");
        }
        // Per-call scratch comes from a pool of the library that keeps what it
        // has reserved (a release threshold of 0, the default pool's, would
        // return freed memory at every synchronisation and make the next
        // allocation map it again).
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        e = cudaMemPoolCreate(&n.pool, &props);
        if (e != cudaSuccess) {
            cudaFree(n.d_status);
            return cuda_fail(e, "cudaMemPoolCreate");
        }
        uint64_t keep = ~uint64_t(0);
        e = cudaMemPoolSetAttribute(n.pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(n.pool);
            cudaFree(n.d_status);
            return cuda_fail(e, "cudaMemPoolSetAttribute");
        }
        d = n;
    }
    *out = d;
    return SDF_OK;
}

// Device memory of `dev` (device or managed allocation) or fails with SDF_ERR_ARG.
int check_device_ptr(const void* p, int dev, const char* name) {
    if (p == nullptr) return fail(SDF_ERR_ARG, "%s is NULL", name);
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SDF_ERR_ARG, "%s: not a CUDA pointer (%s)", name, cudaGetErrorString(e));
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return fail(SDF_ERR_ARG, "%s must be device memory", name);
    if (at.type == cudaMemoryTypeDevice && at.device != dev)
        return fail(SDF_ERR_ARG, "%s lives on device %d, the network on device %d", name, at.device, dev);
    return SDF_OK;
}

uint32_t rd_u32(const uint8_t* p) {
    return static_cast<uint32_t>(p[0]) | (static_cast<uint32_t>(p[1]) << 8) | (static_cast<uint32_t>(p[2]) << 16) |
           (static_cast<uint32_t>(p[3]) << 24);
}
float rd_f32(const uint8_t* p) {
    const uint32_t u = rd_u32(p);
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// Largest singular value by power iteration on M^T M in double precision.
double top_singular_value(const std::vector<double>& M, int rows, int cols) {
    std::vector<double> x(cols, 1.0), y(rows);
    double prev = 0.0;
    for (int it = 0; it < 200000; ++it) {
        double nx = 0.0;
        for (double v : x) nx += v * v;
        nx = std::sqrt(nx);
        if (nx == 0.0) return 0.0;
        for (double& v : x) v /= nx;
        for (int r = 0; r < rows; ++r) {
            double s = 0.0;
            const double* row = &M[static_cast<size_t>(r) * cols];
            for (int c = 0; c < cols; ++c) s += row[c] * x[c];
            y[r] = s;
        }
        double ny = 0.0;
        for (double v : y) ny += v * v;
        const double sigma = std::sqrt(ny);
        std::fill(x.begin(), x.end(), 0.0);
        for (int r = 0; r < rows; ++r) {
            const double* row = &M[static_cast<size_t>(r) * cols];
            for (int c = 0; c < cols; ++c) x[c] += row[c] * y[r];
        }
        if (it > 16 && std::fabs(sigma - prev) <= 1e-15 * sigma) return sigma;
        prev = sigma;
    }
    return prev;
}

uint16_t to_bf16_rne(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return static_cast<uint16_t>(u >> 16);
    u += 0x7fffu + ((u >> 16) & 1u);
    return static_cast<uint16_t>(u >> 16);
}

// E4M3: 1 sign bit, 4 exponent bits (bias 7), 3 mantissa bits; subnormals
// below 2^-6 with spacing 2^-9; largest finite value 448; no infinities.
// Rounds to nearest even and saturates to +-448.
uint8_t to_e4m3(double x) {
    const uint8_t sign = std::signbit(x) ? 0x80u : 0u;
    const double a = std::fabs(x);
    if (std::isnan(a)) return sign | 0x7Fu;
    if (a >= 448.0) return sign | 0x7Eu;
    int e = 0;
    std::frexp(a, &e);
    int E = std::max(e - 1, -6);                            // a in [2^E, 2^(E+1)) for normals
    const double r = std::nearbyint(std::ldexp(a, 3 - E));  // multiples of the spacing 2^(E-3)
    int code;
    if (r < 8.0)
        code = static_cast<int>(r);                          // subnormal (E = -6)
    else if (r < 16.0)
        code = ((E + 7) << 3) | (static_cast<int>(r) - 8);
    else
        code = (E + 8) << 3;                                 // rounded up to the next binade
    return sign | static_cast<uint8_t>(std::min(code, 0x7E));
}

double from_e4m3(uint8_t c) {
    const int biased = (c >> 3) & 15, mant = c & 7;
    const double v = biased == 0 ? std::ldexp(mant, -9) : std::ldexp(8 + mant, biased - 10);
    return (c & 0x80u) ? -v : v;
}

// Largest |G_l| (tangents of Alg. 2 after layer l, over the three spatial
// directions and all units) at a 7 x 7 x 7 grid of points spanning the cube
// [-1, 1]^3 (time 0.5 for 4-input networks), in FP64.
void tangent_maxima(const std::vector<std::vector<double>>& Wl, const std::vector<std::vector<double>>& bl, int IN,
                    int W, int KH, double* out) {
    for (int l = 0; l <= KH; ++l) out[l] = 0.0;
    std::vector<double> P(W), G(3 * W), A(W), Pn(W), Gn(3 * W);
    for (int gi = 0; gi < 343; ++gi) {
        const double x[4] = {-1.0 + (gi % 7) / 3.0, -1.0 + (gi / 7 % 7) / 3.0, -1.0 + (gi / 49) / 3.0, 0.5};
        for (int i = 0; i < W; ++i) {
            double z = bl[0][i];
            for (int c = 0; c < IN; ++c) z += Wl[0][static_cast<size_t>(i) * IN + c] * x[c];
            P[i] = std::sin(z);
            for (int c = 0; c < 3; ++c) {
                G[c * W + i] = Wl[0][static_cast<size_t>(i) * IN + c] * std::cos(z);
                out[0] = std::max(out[0], std::fabs(G[c * W + i]));
            }
        }
        for (int l = 1; l <= KH; ++l) {
            for (int i = 0; i < W; ++i) {
                const double* row = &Wl[l][static_cast<size_t>(i) * W];
                double z = bl[l][i], g[3] = {0.0, 0.0, 0.0};
                for (int k = 0; k < W; ++k) {
                    z += row[k] * P[k];
                    for (int c = 0; c < 3; ++c) g[c] += row[k] * G[c * W + k];
                }
                Pn[i] = std::sin(z);
                const double cz = std::cos(z);
                for (int c = 0; c < 3; ++c) {
                    Gn[c * W + i] = cz * g[c];
                    out[l] = std::max(out[l], std::fabs(Gn[c * W + i]));
                }
            }
            P.swap(Pn);
            G.swap(Gn);
        }
    }
}

NetView view_of(const sdf_net* n) {
    NetView v{};
    v.in_dim = n->in_dim;
    v.width = n->width;
    v.n_hidden = n->n_hidden;
    v.w0 = n->d_f32 + n->off_w0;
    v.b0 = n->d_f32 + n->off_b0;
    for (int l = 0; l < n->n_hidden; ++l) {
        v.wt[l] = n->d_f32 + n->off_wt[l];
        v.bh[l] = n->d_f32 + n->off_bh[l];
    }
    v.wout = n->d_f32 + n->off_wout;
    v.bout = n->bout;
    v.wbf = n->d_bf16;
    v.wbf_lo = n->d_bf16 ? n->d_bf16 + static_cast<size_t>(n->n_hidden) * n->bf16_layer_bytes : nullptr;
    v.wbf_layer_bytes = n->bf16_layer_bytes;
    v.rows_pad = n->rows_pad;
    v.op_f16 = n->precision == SDF_FP16 ? 1 : 0;
    if (n->precision == SDF_FP8) {
        v.op_fp8 = 1;
        v.wbf_lo = nullptr;
        for (int l = 0; l < n->n_hidden; ++l) v.q_w[l] = n->q_w[l];
        for (int l = 0; l <= n->n_hidden; ++l) v.q_g[l] = n->q_g[l];
        v.q_o = n->q_o;
        v.wout_q = n->d_bf16 + static_cast<size_t>(n->n_hidden) * n->bf16_layer_bytes;
    }
    return v;
}

void free_net(sdf_net* n) {
    if (!n) return;
    DeviceGuard g(n->device);
    if (n->d_f32) cudaFree(n->d_f32);
    if (n->d_bf16) cudaFree(n->d_bf16);
    delete n;
}

// An SDFN image parsed on the host: shape and the folded parameters of
// Eq. 2 in FP64 (layer 0 multiplied by omega0, hidden layers by omega, the
// output layer unchanged), so every sine layer reads plain sin(W x + b).
struct ParsedImage {
    int IN = 0, W = 0, KH = 0;
    std::vector<std::vector<double>> Wl, bl;  // layers 0..KH: [W][fan_in] row-major, [W]
    std::vector<double> wout;
    float bout = 0.0f;
};

// Parses and folds an SDFN image; checks the header, the size and that every
// parameter is finite (shape support is the caller's business).
int parse_image(const uint8_t* buf, size_t len, ParsedImage* P) {
    if (!buf) return fail(SDF_ERR_ARG, "bytes is NULL");
    if (len < 32 || std::memcmp(buf, "SDFN", 4) != 0) return fail(SDF_ERR_FORMAT, "not an SDFN image");
    const uint32_t version = rd_u32(buf + 4), in_dim = rd_u32(buf + 8), width = rd_u32(buf + 12);
    const uint32_t n_hidden = rd_u32(buf + 16), flags = rd_u32(buf + 28);
    const float omega0 = rd_f32(buf + 20), omega = rd_f32(buf + 24);
    if (version != 1) return fail(SDF_ERR_FORMAT, "unsupported SDFN version %u", version);
    if (in_dim < 1 || in_dim > 4096 || width < 1 || width > 4096 || n_hidden > 64)
        return fail(SDF_ERR_FORMAT, "implausible shape in=%u width=%u hidden=%u", in_dim, width, n_hidden);
    const size_t count = static_cast<size_t>(width) * in_dim + width +
                         static_cast<size_t>(n_hidden) * (static_cast<size_t>(width) * width + width) + width + 1;
    if (len != 32 + 4 * count) return fail(SDF_ERR_FORMAT, "SDFN size %zu, expected %zu", len, 32 + 4 * count);
    if (!std::isfinite(omega0) || !std::isfinite(omega)) return fail(SDF_ERR_NONFINITE, "non-finite omega");
    const uint8_t* q = buf + 32;
    for (size_t i = 0; i < count; ++i)
        if (!std::isfinite(rd_f32(q + 4 * i))) return fail(SDF_ERR_NONFINITE, "non-finite parameter %zu", i);
    const int W = static_cast<int>(width), IN = static_cast<int>(in_dim), KH = static_cast<int>(n_hidden);
    const bool folded = (flags & 1u) != 0;
    P->IN = IN;
    P->W = W;
    P->KH = KH;
    P->Wl.assign(KH + 1, {});
    P->bl.assign(KH + 1, {});
    size_t o = 0;
    for (int l = 0; l <= KH; ++l) {
        const int fan_in = l == 0 ? IN : W;
        const double s = folded ? 1.0 : (l == 0 ? omega0 : omega);
        P->Wl[l].resize(static_cast<size_t>(W) * fan_in);
        P->bl[l].resize(W);
        for (auto& v : P->Wl[l]) v = s * rd_f32(q + 4 * o++);
        for (auto& v : P->bl[l]) v = s * rd_f32(q + 4 * o++);
    }
    P->wout.resize(W);
    for (auto& v : P->wout) v = rd_f32(q + 4 * o++);
    P->bout = rd_f32(q + 4 * o++);
    return SDF_OK;
}

int load_from_memory(const uint8_t* buf, size_t len, int precision, int device, sdf_net_t* out) {
    if (!out) return fail(SDF_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!buf) return fail(SDF_ERR_ARG, "bytes is NULL");
    if (precision != SDF_FP32 && precision != SDF_BF16 && precision != SDF_FP16 && precision != SDF_FP8)
        return fail(SDF_ERR_ARG, "unknown precision %d", precision);
    ParsedImage img;
    int rc = parse_image(buf, len, &img);
    if (rc) return rc;
    if ((img.IN != 3 && img.IN != 4) || (img.W != 64 && img.W != 128 && img.W != 256) || img.KH < 1 ||
        img.KH > kMaxHidden)
        return fail(SDF_ERR_UNSUPPORTED, "shape in=%d (w=%d, k=%d) not supported (in 3|4, w 64|128|256, 1<=k<=%d)",
                    img.IN, img.W, img.KH, kMaxHidden);
    if (precision == SDF_FP8 && img.W < 128)
        return fail(SDF_ERR_UNSUPPORTED, "E4M3 hidden layers need width 128 or 256 (got %d)", img.W);
    const int W = img.W, IN = img.IN, KH = img.KH;
    const std::vector<std::vector<double>>& Wl = img.Wl;
    const std::vector<std::vector<double>>& bl = img.bl;
    const std::vector<double>& wout = img.wout;
    const float bout = img.bout;

    // Lipschitz bound of Eq. 2 (sin is 1-Lipschitz)
    double L = top_singular_value(Wl[0], W, IN);
    for (int l = 1; l <= KH; ++l) L *= top_singular_value(Wl[l], W, W);
    double nw = 0.0;
    for (double v : wout) nw += v * v;
    L *= std::sqrt(nw);

    sdf_net* n = new sdf_net;
    n->device = device;
    n->precision = precision;
    n->in_dim = IN;
    n->width = W;
    n->n_hidden = KH;
    n->lipschitz = L;
    n->bout = bout;

    // FP32 layout: w0 [W][IN], b0, then per hidden layer W^T [k][n] and b, then w_out
    std::vector<float> f32;
    n->off_w0 = f32.size();
    for (double v : Wl[0]) f32.push_back(static_cast<float>(v));
    n->off_b0 = f32.size();
    for (double v : bl[0]) f32.push_back(static_cast<float>(v));
    for (int l = 1; l <= KH; ++l) {
        while (f32.size() % 4) f32.push_back(0.0f);
        n->off_wt[l - 1] = f32.size();
        for (int k = 0; k < W; ++k)
            for (int r = 0; r < W; ++r) f32.push_back(static_cast<float>(Wl[l][static_cast<size_t>(r) * W + k]));
        n->off_bh[l - 1] = f32.size();
        for (double v : bl[l]) f32.push_back(static_cast<float>(v));
    }
    n->off_wout = f32.size();
    for (double v : wout) f32.push_back(static_cast<float>(v));

    // 16-bit hidden weights (bfloat16 or half, round to nearest even), K-major
    // with the 128-byte swizzle, rows padded to >= 128
    std::vector<uint8_t> bf;
    if (precision == SDF_BF16 || precision == SDF_FP16) {
        // heads for all layers, then the remainders (weight - head) rounded again
        n->rows_pad = W < 128 ? 128 : W;
        n->bf16_layer_bytes = static_cast<uint32_t>(n->rows_pad) * W * 2u;
        const size_t half_bytes = static_cast<size_t>(KH) * n->bf16_layer_bytes;
        bf.assign(2 * half_bytes, 0);
        auto to16 = [&](float x) -> uint16_t {
            return precision == SDF_FP16 ? __half_as_ushort(__float2half_rn(x)) : to_bf16_rne(x);
        };
        auto from16 = [&](uint16_t h) -> float {
            if (precision == SDF_FP16) return __half2float(__ushort_as_half(h));
            const uint32_t u = static_cast<uint32_t>(h) << 16;
            float f;
            std::memcpy(&f, &u, 4);
            return f;
        };
        for (int l = 1; l <= KH; ++l) {
            uint8_t* dst = bf.data() + static_cast<size_t>(l - 1) * n->bf16_layer_bytes;
            for (int r = 0; r < W; ++r)
                for (int k = 0; k < W; ++k) {
                    const float x = static_cast<float>(Wl[l][static_cast<size_t>(r) * W + k]);
                    const uint16_t h = to16(x);
                    const uint16_t lo = to16(x - from16(h));
                    std::memcpy(dst + sw128_offset(r, k, n->rows_pad), &h, 2);
                    std::memcpy(dst + half_bytes + sw128_offset(r, k, n->rows_pad), &lo, 2);
                }
        }
    }

    // E4M3 hidden weights with per-layer scales 448 / max|W_l|, K-major with the
    // 128-byte swizzle (128-element K blocks); then the output row as head and
    // remainder; tangent scales from the calibration grid (largest |G_l| -> 64)
    if (precision == SDF_FP8) {
        n->rows_pad = W;
        n->bf16_layer_bytes = static_cast<uint32_t>(W) * W;
        bf.assign(static_cast<size_t>(KH) * n->bf16_layer_bytes + 2 * static_cast<size_t>(W), 0);
        for (int l = 1; l <= KH; ++l) {
            double amax = 0.0;
            for (double v : Wl[l]) amax = std::max(amax, std::fabs(v));
            const double qw = amax > 0.0 ? 448.0 / amax : 1.0;
            n->q_w[l - 1] = static_cast<float>(qw);
            uint8_t* dst = bf.data() + static_cast<size_t>(l - 1) * n->bf16_layer_bytes;
            for (int r = 0; r < W; ++r)
                for (int k = 0; k < W; ++k)
                    dst[sw128_offset8(r, k, W)] = to_e4m3(Wl[l][static_cast<size_t>(r) * W + k] * qw);
        }
        double amax = 0.0;
        for (double v : wout) amax = std::max(amax, std::fabs(v));
        const double qo = amax > 0.0 ? 448.0 / amax : 1.0;
        n->q_o = static_cast<float>(qo);
        uint8_t* wq = bf.data() + static_cast<size_t>(KH) * n->bf16_layer_bytes;
        for (int k = 0; k < W; ++k) {
            const uint8_t hd = to_e4m3(wout[k] * qo);
            wq[k] = hd;
            wq[W + k] = to_e4m3((wout[k] * qo - from_e4m3(hd)) * 16.0);
        }
        double gmax[kMaxHidden + 1];
        tangent_maxima(Wl, bl, IN, W, KH, gmax);
        for (int l = 0; l <= KH; ++l) n->q_g[l] = static_cast<float>(gmax[l] > 0.0 ? 64.0 / gmax[l] : 1.0);
    }

    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        delete n;
        return fail(SDF_ERR_ARG, "device %d not available", device);
    }
    DeviceGuard g(device);
    if (!g.ok) {
        delete n;
        return fail(SDF_ERR_CUDA, "cudaSetDevice(%d) failed", device);
    }
    cudaError_t e = cudaMalloc(&n->d_f32, f32.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(n->d_f32, f32.data(), f32.size() * sizeof(float), cudaMemcpyHostToDevice);
    n->h_f32 = f32;
    if (e == cudaSuccess && !bf.empty()) {
        e = cudaMalloc(&n->d_bf16, bf.size());
        if (e == cudaSuccess) e = cudaMemcpy(n->d_bf16, bf.data(), bf.size(), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        free_net(n);
        return cuda_fail(e, "uploading network");
    }
    *out = n;
    g_last_error.clear();
    return SDF_OK;
}

bool finite_pos(float x) { return std::isfinite(x) && x > 0.0f; }

struct Scratch {
    void* ptr = nullptr;
    cudaStream_t s = nullptr;
    ~Scratch() {
        if (ptr) cudaFreeAsync(ptr, s);
    }
};

// Checks the parameters and buffers of a trace; *dev receives the device of
// the networks.  Device pointers are checked only when n > 0.
int validate_trace_params(const sdf_trace_params* P, int* dev_out) {
    if (!P) return fail(SDF_ERR_ARG, "params is NULL");
    const int m = P->n_levels;
    if (m < 1 || m > kMaxLevels) return fail(SDF_ERR_ARG, "n_levels = %d out of range 1..%d", m, kMaxLevels);
    if (!P->nets || !P->delta || !P->max_iters) return fail(SDF_ERR_ARG, "nets, delta and max_iters are required");
    if (!finite_pos(P->eps)) return fail(SDF_ERR_ARG, "eps must be finite and > 0");
    if (!std::isfinite(P->box_min) || !std::isfinite(P->box_max) || !(P->box_min < P->box_max))
        return fail(SDF_ERR_ARG, "box_min < box_max required");
    if (P->final_mode != 0 && P->final_mode != 1) return fail(SDF_ERR_ARG, "final_mode must be 0 or 1");
    if (!std::isfinite(P->time)) return fail(SDF_ERR_ARG, "time must be finite");
    const int dev = P->nets[0] ? P->nets[0]->device : -1;
    for (int j = 0; j < m; ++j) {
        const sdf_net* net = P->nets[j];
        if (!net) return fail(SDF_ERR_ARG, "nets[%d] is NULL", j);
        if (net->device != dev) return fail(SDF_ERR_ARG, "networks live on different devices");
        if (net->in_dim != P->nets[0]->in_dim) return fail(SDF_ERR_ARG, "networks differ in input dimension");
        if (P->max_iters[j] < 0) return fail(SDF_ERR_ARG, "max_iters[%d] < 0", j);
        const bool uses_delta = (j < m - 1) || P->final_mode == 1;
        if (uses_delta && !finite_pos(P->delta[j])) return fail(SDF_ERR_ARG, "delta[%d] must be finite and > 0", j);
        if (P->step_scale && !finite_pos(P->step_scale[j]))
            return fail(SDF_ERR_ARG, "step_scale[%d] must be finite and > 0", j);
        if (!P->step_scale && !(net->lipschitz > 0.0))
            return fail(SDF_ERR_ARG, "nets[%d] has a zero Lipschitz bound; pass step_scale", j);
        if (net->precision == SDF_FP8 && net->width != 256)
            return fail(SDF_ERR_UNSUPPORTED, "nets[%d]: tracing with E4M3 hidden layers is built for width 256", j);
        if (net->precision != SDF_FP32 && !tc_trace_supported(net->width, net->n_hidden))
            return fail(SDF_ERR_UNSUPPORTED, "tensor-core tracing of a (%d,%d) network is not built", net->width,
                        net->n_hidden);
    }
    if (P->ray_time && P->nets[0]->in_dim != 4) return fail(SDF_ERR_ARG, "ray_time given for 3-input networks");
    *dev_out = dev;
    return SDF_OK;
}

int validate_trace(const sdf_trace_params* P, const float* orig, const float* dir, int64_t n, const float* out_pos,
                   const float* out_t, const uint8_t* out_hit, const uint16_t* out_iters, int* dev_out) {
    if (!P) return fail(SDF_ERR_ARG, "params is NULL");
    if (n < 0 || n > 0x7fffffffLL) return fail(SDF_ERR_ARG, "n = %lld out of range", static_cast<long long>(n));
    int rc = validate_trace_params(P, dev_out);
    if (rc) return rc;
    const int dev = *dev_out;
    if (n == 0) return SDF_OK;
    DeviceGuard g(dev);
    if (!g.ok) return fail(SDF_ERR_CUDA, "cudaSetDevice(%d) failed", dev);
    if ((rc = check_device_ptr(orig, dev, "orig")) || (rc = check_device_ptr(dir, dev, "dir")) ||
        (rc = check_device_ptr(out_pos, dev, "out_pos")) || (rc = check_device_ptr(out_t, dev, "out_t")) ||
        (rc = check_device_ptr(out_hit, dev, "out_hit")))
        return rc;
    if (out_iters && (rc = check_device_ptr(out_iters, dev, "out_iters"))) return rc;
    if (P->ray_time && (rc = check_device_ptr(P->ray_time, dev, "ray_time"))) return rc;
    return SDF_OK;
}

// Bytes of trace scratch: 2 * kMaxLevels counters (grab_j, count_j), then
// two ray-index queues of n entries when there is more than one level.
size_t trace_scratch_bytes(int m, int64_t n) {
    return 2 * kMaxLevels * sizeof(unsigned long long) + ((m > 1) ? 2 * static_cast<size_t>(n) * sizeof(int32_t) : 0);
}

// The width-64 parameters of one level as launch parameters (TraceConsts):
// the same values, in the same pair layout, as the kernel would otherwise
// stage in shared memory, the scalar time folded into the layer-0 bias by
// one fused multiply-add as there.
void fill_trace_consts(const sdf_net* n, LevelArgs& la) {
    const float* f = n->h_f32.data();
    const float *w0 = f + n->off_w0, *b0 = f + n->off_b0, *bl = f + n->off_bh[n->n_hidden - 1], *wo = f + n->off_wout;
    const bool timed = la.ray_time != nullptr && n->in_dim == 4;
    float* bls = &la.k.bl[0].x;
    float* wos = &la.k.wo[0].x;
    for (int i = 0; i < kConstWidth; ++i) {
        const int p = i >> 1, e = i & 1;
        const float wt = n->in_dim == 4 ? w0[i * 4 + 3] : 0.0f;
        const float bb = timed ? b0[i] : std::fma(wt, la.time, b0[i]);
        float* pa = &la.k.w0[2 * p].x;
        float* pb = &la.k.w0[2 * p + 1].x;
        pa[e] = w0[i * n->in_dim + 0];
        pa[2 + e] = w0[i * n->in_dim + 1];
        pb[e] = w0[i * n->in_dim + 2];
        pb[2 + e] = bb;
        bls[i] = bl[i];
        wos[i] = wo[i];
    }
}

// Zeroes the 2 * kMaxLevels counters and launches the levels of Alg. 1 on
// `s` (the validated parameters' device current); list0 / list1 hold n
// entries each (unused with one level).  tiles: per-level tile counts for
// the tensor-core kernel, or NULL.
int launch_levels_at(const sdf_trace_params* P, const float* orig, const float* dir, int64_t n, float* out_pos,
                     float* out_t, uint8_t* out_hit, uint16_t* out_iters, unsigned long long* counters,
                     int32_t* list0, int32_t* list1, int* status, int num_sms, const int* tiles, cudaStream_t s) {
    const int m = P->n_levels;
    cudaError_t e = cudaMemsetAsync(counters, 0, 2 * kMaxLevels * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(counters)");
    int32_t* lists[2] = {list0, list1};
    for (int j = 0; j < m; ++j) {
        const sdf_net* net = P->nets[j];
        const bool last = (j == m - 1);
        LevelArgs la{};
        la.net = view_of(net);
        la.d = (last && P->final_mode == 0) ? 0.0f : P->delta[j];
        la.scale = P->step_scale ? P->step_scale[j] : static_cast<float>(1.0 / net->lipschitz);
        la.cap = P->max_iters[j];
        la.is_last = last ? 1 : 0;
        la.time = P->time;
        la.ray_time = P->ray_time;
        la.tiles = tiles ? tiles[j] : 0;
        la.eps = P->eps;
        la.box_lo = P->box_min;
        la.box_hi = P->box_max;
        la.orig = orig;
        la.dir = dir;
        la.n = n;
        la.out_pos = out_pos;
        la.out_t = out_t;
        la.out_hit = out_hit;
        la.out_iters = out_iters;
        la.in_list = j == 0 ? nullptr : lists[(j - 1) & 1];
        la.in_count = j == 0 ? nullptr : &counters[kMaxLevels + j - 1];
        la.out_list = last ? nullptr : lists[j & 1];
        la.out_count = last ? nullptr : &counters[kMaxLevels + j];
        la.grab = &counters[j];
        la.status = status;
        if (net->width == kConstWidth) fill_trace_consts(net, la);
        e = (net->precision != SDF_FP32) ? launch_trace_level_tc(la, num_sms, s)
                                         : launch_trace_level_simt(la, num_sms, s);
        if (e != cudaSuccess) return cuda_fail(e, "launching trace level");
    }
    return SDF_OK;
}

// launch_levels_at with the counters and queues laid out in one block of
// trace_scratch_bytes(m, n) bytes.
int launch_levels(const sdf_trace_params* P, const float* orig, const float* dir, int64_t n, float* out_pos,
                  float* out_t, uint8_t* out_hit, uint16_t* out_iters, void* scratch, int* status, int num_sms,
                  const int* tiles, cudaStream_t s) {
    auto* counters = static_cast<unsigned long long*>(scratch);
    int32_t* l0 = reinterpret_cast<int32_t*>(counters + 2 * kMaxLevels);
    return launch_levels_at(P, orig, dir, n, out_pos, out_t, out_hit, out_iters, counters, l0, l0 + n, status,
                            num_sms, tiles, s);
}

int trace_impl(const sdf_trace_params* P, const float* orig, const float* dir, int64_t n, float* out_pos,
               float* out_t, uint8_t* out_hit, uint16_t* out_iters, cudaStream_t s) {
    int dev = -1;
    int rc = validate_trace(P, orig, dir, n, out_pos, out_t, out_hit, out_iters, &dev);
    if (rc || n == 0) return rc;
    DeviceGuard g(dev);
    if (!g.ok) return fail(SDF_ERR_CUDA, "cudaSetDevice(%d) failed", dev);
    DeviceInfo di;
    if ((rc = device_info(dev, &di))) return rc;
    Scratch sc;
    sc.s = s;
    cudaError_t e = cudaMallocFromPoolAsync(&sc.ptr, trace_scratch_bytes(P->n_levels, n) + 256, di.pool, s);
    if (e != cudaSuccess) return cuda_fail(e, "allocating scratch");
    return launch_levels(P, orig, dir, n, out_pos, out_t, out_hit, out_iters, sc.ptr, di.d_status, di.num_sms,
                         nullptr, s);
}

// Checks a gradient / normal-map call (the network's device current when n > 0).
int validate_grad(sdf_net_t net, const float* pts, const float* pt_time, const uint8_t* mask, int64_t n,
                  const float* out) {
    if (!net) return fail(SDF_ERR_ARG, "net is NULL");
    if (n < 0 || n > 0x7fffffffLL) return fail(SDF_ERR_ARG, "n = %lld out of range", static_cast<long long>(n));
    if (pt_time && net->in_dim != 4) return fail(SDF_ERR_ARG, "per-point times given for a 3-input network");
    if (net->precision != SDF_FP32 && !tc_grad_supported(net->width, net->n_hidden))
        return fail(SDF_ERR_UNSUPPORTED, "tensor-core gradients of a (%d,%d) network are not built", net->width,
                    net->n_hidden);
    if (n == 0) return SDF_OK;
    int rc;
    if ((rc = check_device_ptr(pts, net->device, "pts")) || (rc = check_device_ptr(out, net->device, "out")))
        return rc;
    if (mask && (rc = check_device_ptr(mask, net->device, "mask"))) return rc;
    if (pt_time && (rc = check_device_ptr(pt_time, net->device, "time"))) return rc;
    return SDF_OK;
}

// Bytes of gradient scratch: 4 counters, then a list of n indices with a mask.
size_t grad_scratch_bytes(int64_t n, bool mask) {
    return 4 * sizeof(unsigned long long) + (mask ? static_cast<size_t>(n) * sizeof(int32_t) : 0);
}

// With a mask, the entries it excludes are zeroed in `out` by the compaction
// kernel unless zero_unmasked is false (the caller zeroes them itself).
int launch_gradients(sdf_net_t net, const float* pts, const float* pt_time, const uint8_t* mask, int64_t n, float* out,
                     int normalize, void* scratch, int* status, int num_sms, cudaStream_t s,
                     bool zero_unmasked = true) {
    const size_t counter_bytes = 4 * sizeof(unsigned long long);
    cudaError_t e = cudaMemsetAsync(scratch, 0, counter_bytes, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(counters)");
    auto* counters = static_cast<unsigned long long*>(scratch);
    int32_t* list = mask ? reinterpret_cast<int32_t*>(static_cast<uint8_t*>(scratch) + counter_bytes) : nullptr;
    if (mask) {
        e = launch_mask_compact(mask, n, list, &counters[1], zero_unmasked ? out : nullptr, num_sms, s);
        if (e != cudaSuccess) return cuda_fail(e, "launching mask compaction");
    }
    GradArgs ga{};
    ga.net = view_of(net);
    ga.time = net->time;
    ga.pt_time = pt_time;
    ga.pts = pts;
    ga.n = n;
    ga.list = list;
    ga.count = mask ? &counters[1] : nullptr;
    ga.out = out;
    ga.normalize = normalize;
    ga.grab = &counters[0];
    ga.status = status;
    e = (net->precision != SDF_FP32) ? launch_grad_tc(ga, num_sms, s) : launch_grad_simt(ga, num_sms, s);
    if (e != cudaSuccess) return cuda_fail(e, "launching gradient kernel");
    return SDF_OK;
}

int grad_impl(sdf_net_t net, const float* pts, const float* pt_time, const uint8_t* mask, int64_t n, float* out,
              int normalize, cudaStream_t s) {
    if (!net) return fail(SDF_ERR_ARG, "net is NULL");
    DeviceGuard g(net->device);
    if (!g.ok) return fail(SDF_ERR_CUDA, "cudaSetDevice(%d) failed", net->device);
    int rc = validate_grad(net, pts, pt_time, mask, n, out);
    if (rc || n == 0) return rc;
    DeviceInfo di;
    if ((rc = device_info(net->device, &di))) return rc;
    Scratch sc;
    sc.s = s;
    cudaError_t e = cudaMallocFromPoolAsync(&sc.ptr, grad_scratch_bytes(n, mask != nullptr) + 256, di.pool, s);
    if (e != cudaSuccess) return cuda_fail(e, "allocating scratch");
    return launch_gradients(net, pts, pt_time, mask, n, out, normalize, sc.ptr, di.d_status, di.num_sms, s);
}

}  // namespace

// ---------------------------------------------------------------------------
// Scratch for sdf_trace_multiscale_noalloc: work counters, a status word and
// the two ray-index queues between levels, for at most kNoAllocMaxRays rays.
// It is a static device array, so it exists on every device that loads this
// library, from module load until the process exits (16 MB + 256 bytes).
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t kNoAllocMaxRays = int64_t(1) << 21;  // 2,097,152 rays: one 1920 x 1080 frame fits

struct NoAllocLayout {
    unsigned long long counters[2 * kMaxLevels];  // grab_j, count_j; zeroed at the start of every call
    int status;                                   // device-side timeouts of this entry point
    int pad[63];
    int32_t lists[2][kNoAllocMaxRays];            // ping-pong ray-index queues between levels
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocLayout)];

struct NoAllocDevice {
    bool ready = false;
    int num_sms = 0;
    NoAllocLayout* scratch = nullptr;  // device address of g_noalloc_scratch on this device
};

std::mutex g_noalloc_mutex;
NoAllocDevice g_noalloc_dev[64];

// Device address of the static scratch and the SM count of `dev`, looked up
// once per device with that device current.  Allocates nothing.
int noalloc_setup(int dev, NoAllocDevice* out) {
    if (dev < 0 || dev >= 64) return fail(SDF_ERR_ARG, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    NoAllocDevice& d = g_noalloc_dev[dev];
    if (!d.ready) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
        e = cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
        d.scratch = static_cast<NoAllocLayout*>(p);
        d.ready = true;
    }
    *out = d;
    return SDF_OK;
}

// Reads and clears the status word of the static scratch on `dev` (the
// caller has made `dev` current).  *status is 0 when no call of the
// allocation-free entry point has set the array up on this device.
int noalloc_take_status(int dev, int* status) {
    *status = 0;
    if (dev < 0 || dev >= 64) return SDF_OK;
    NoAllocLayout* sc = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_dev[dev].ready) return SDF_OK;
        sc = g_noalloc_dev[dev].scratch;
    }
    cudaError_t e = cudaMemcpy(status, &sc->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading the status word of the static scratch");
    if (*status != 0) {
        const int zero = 0;
        e = cudaMemcpy(&sc->status, &zero, sizeof(int), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "clearing the status word of the static scratch");
    }
    return SDF_OK;
}

}  // namespace


// ---------------------------------------------------------------------------
// Frame-batch plans: one CUDA graph holding the whole trace (all levels) and
// the normal-mapping stage for a fixed set of device buffers.
// ---------------------------------------------------------------------------
struct sdf_plan {
    int device = 0;
    int n_levels = 0;
    sdf_net_t nets[kMaxLevels] = {};
    float delta[kMaxLevels] = {}, step_scale[kMaxLevels] = {};
    int max_iters[kMaxLevels] = {}, tiles[kMaxLevels] = {};
    sdf_trace_params params{};  // points into the arrays above
    sdf_net_t fine = nullptr;
    sdf_frame_batch batch{};
    void* scratch = nullptr;    // trace scratch, then gradient scratch
    size_t trace_bytes = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t n_nodes = 0;
};

namespace {

void free_plan(sdf_plan* p) {
    if (!p) return;
    DeviceGuard g(p->device);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->scratch) cudaFree(p->scratch);
    delete p;
}

// Every launch of the plan's work on `s` (also what the graph captures).
int plan_enqueue(sdf_plan* p, const int* tiles, int* status, int num_sms, cudaStream_t s) {
    const sdf_frame_batch& b = p->batch;
    int rc = launch_levels(&p->params, b.orig, b.dir, b.n, b.out_pos, b.out_t, b.out_hit, b.out_iters, p->scratch,
                           status, num_sms, tiles, s);
    if (rc || !p->fine) return rc;
    return launch_gradients(p->fine, b.out_pos, b.ray_time, b.out_hit, b.n, b.out_normal, 1,
                            static_cast<uint8_t*>(p->scratch) + p->trace_bytes, status, num_sms, s);
}

// Coordinate search over the tile count of each tensor-core level: for
// level j every count 1..maximum is timed on the plan's own buffers (the
// whole trace, one warm-up and the best of two runs) with the counts already
// chosen for levels < j, and the fastest is kept.
int plan_autotune(sdf_plan* p, int* status, int num_sms, cudaStream_t s) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(e, "cudaEventCreate");
    }
    int rc = SDF_OK;
    const sdf_frame_batch& b = p->batch;
    for (int j = 0; j < p->n_levels && rc == SDF_OK; ++j) {
        const sdf_net* net = p->nets[j];
        const int tmax = net->precision == SDF_FP32 ? 0 : trace_tiles_max(view_of(net));
        if (tmax <= 1) continue;
        float best = INFINITY;
        int best_t = tmax;
        for (int t = 1; t <= tmax && rc == SDF_OK; ++t) {
            p->tiles[j] = t;
            float ms_min = INFINITY;
            for (int rep = 0; rep < 3 && rc == SDF_OK; ++rep) {
                cudaEventRecord(e0, s);
                rc = launch_levels(&p->params, b.orig, b.dir, b.n, b.out_pos, b.out_t, b.out_hit, b.out_iters,
                                   p->scratch, status, num_sms, p->tiles, s);
                cudaEventRecord(e1, s);
                if ((e = cudaEventSynchronize(e1)) != cudaSuccess) rc = cuda_fail(e, "autotune run");
                float ms = 0.0f;
                if (rc == SDF_OK && rep > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
                    ms_min = std::min(ms_min, ms);
            }
            if (ms_min < best) {
                best = ms_min;
                best_t = t;
            }
        }
        p->tiles[j] = best_t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

int plan_create(const sdf_trace_params* P, sdf_net_t fine, const sdf_frame_batch* B, int autotune,
                cudaStream_t s, sdf_plan_t* out) {
    if (!out) return fail(SDF_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!B) return fail(SDF_ERR_ARG, "batch is NULL");
    if (!P) return fail(SDF_ERR_ARG, "params is NULL");
    if (P->ray_time && P->ray_time != B->ray_time)
        return fail(SDF_ERR_ARG, "pass per-ray times in the batch (params->ray_time must be NULL or equal)");
    if ((fine == nullptr) != (B->out_normal == nullptr))
        return fail(SDF_ERR_ARG, "fine and out_normal go together (both or neither)");
    sdf_trace_params Q = *P;
    Q.ray_time = B->ray_time;
    int dev = -1;
    int rc = validate_trace(&Q, B->orig, B->dir, B->n, B->out_pos, B->out_t, B->out_hit, B->out_iters, &dev);
    if (rc) return rc;
    if (fine) {
        if (fine->device != dev) return fail(SDF_ERR_ARG, "fine network on another device");
        if (B->ray_time && fine->in_dim != 4) return fail(SDF_ERR_ARG, "ray_time given for a 3-input fine network");
        DeviceGuard g(dev);
        if ((rc = validate_grad(fine, B->out_pos, B->ray_time, B->out_hit, B->n, B->out_normal))) return rc;
    }
    DeviceGuard g(dev);
    if (!g.ok) return fail(SDF_ERR_CUDA, "cudaSetDevice(%d) failed", dev);
    DeviceInfo di;
    if ((rc = device_info(dev, &di))) return rc;

    sdf_plan* p = new sdf_plan;
    p->device = dev;
    p->n_levels = Q.n_levels;
    for (int j = 0; j < Q.n_levels; ++j) {
        p->nets[j] = Q.nets[j];
        p->delta[j] = Q.delta[j];
        p->max_iters[j] = Q.max_iters[j];
        p->step_scale[j] = Q.step_scale ? Q.step_scale[j] : 0.0f;
    }
    p->params = Q;
    p->params.nets = p->nets;
    p->params.delta = p->delta;
    p->params.max_iters = p->max_iters;
    p->params.step_scale = Q.step_scale ? p->step_scale : nullptr;
    p->fine = fine;
    p->batch = *B;
    if (B->n == 0) {
        *out = p;
        return SDF_OK;
    }
    p->trace_bytes = (trace_scratch_bytes(Q.n_levels, B->n) + 255) & ~size_t(255);
    const size_t grad_bytes = fine ? grad_scratch_bytes(B->n, true) : 0;
    cudaError_t e = cudaMalloc(&p->scratch, p->trace_bytes + grad_bytes + 256);
    if (e != cudaSuccess) {
        free_plan(p);
        return cuda_fail(e, "cudaMalloc(plan scratch)");
    }
    if (autotune && (rc = plan_autotune(p, di.d_status, di.num_sms, s))) {
        free_plan(p);
        return rc;
    }
    // capture on a private stream (the legacy default stream cannot be captured)
    cudaStream_t cs = nullptr;
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) {
        free_plan(p);
        return cuda_fail(e, "cudaStreamCreate");
    }
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        free_plan(p);
        return cuda_fail(e, "cudaStreamBeginCapture");
    }
    rc = plan_enqueue(p, p->tiles, di.d_status, di.num_sms, cs);
    e = cudaStreamEndCapture(cs, &p->graph);
    cudaStreamDestroy(cs);
    if (rc || e != cudaSuccess) {
        if (!rc) rc = cuda_fail(e, "cudaStreamEndCapture");
        free_plan(p);
        return rc;
    }
    if ((e = cudaGraphGetNodes(p->graph, nullptr, &p->n_nodes)) != cudaSuccess ||
        (e = cudaGraphInstantiate(&p->exec, p->graph, 0)) != cudaSuccess) {
        free_plan(p);
        return cuda_fail(e, "instantiating the plan's graph");
    }
    *out = p;
    return SDF_OK;
}

}  // namespace

namespace {

// Streams and events of sdf_render_host on one device (created on first use,
// kept until exit); calls on one device take the mutex for their duration.
constexpr int kHostChunks = 4;
struct HostPipe {
    std::mutex m;
    bool ready = false;
    // copies in, two compute streams (consecutive chunks alternate, so one
    // chunk's kernels fill the SMs its predecessor's tail leaves idle), copies out
    cudaStream_t in = nullptr, cmp[2] = {}, out = nullptr;
    cudaEvent_t start = nullptr, done = nullptr, ev_in[kHostChunks] = {}, ev_cmp[kHostChunks] = {};
};
HostPipe g_host_pipes[64];

int host_pipe_init(HostPipe* hp) {
    if (hp->ready) return SDF_OK;
    cudaError_t e = cudaSuccess;
    for (cudaStream_t* st : {&hp->in, &hp->cmp[0], &hp->cmp[1], &hp->out})
        if (e == cudaSuccess && !*st) e = cudaStreamCreateWithFlags(st, cudaStreamNonBlocking);
    auto mk = [&](cudaEvent_t* ev) {
        if (e == cudaSuccess && !*ev) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    };
    mk(&hp->start);
    mk(&hp->done);
    for (int c = 0; c < kHostChunks; ++c) {
        mk(&hp->ev_in[c]);
        mk(&hp->ev_cmp[c]);
    }
    if (e != cudaSuccess) return cuda_fail(e, "creating the host-frame streams");
    hp->ready = true;
    return SDF_OK;
}

// Device address of [p, p + bytes) when the whole range is page-locked host
// memory mapped into the device's address space (cudaHostAlloc,
// cudaHostRegister, pinned torch tensors), else nullptr.
const void* mapped_host(const void* p, size_t bytes) {
    cudaPointerAttributes a0, a1;
    const void* last = static_cast<const uint8_t*>(p) + (bytes - 1);
    if (cudaPointerGetAttributes(&a0, p) != cudaSuccess || cudaPointerGetAttributes(&a1, last) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a0.type != cudaMemoryTypeHost || a1.type != cudaMemoryTypeHost || !a0.devicePointer || !a1.devicePointer)
        return nullptr;
    if (static_cast<const uint8_t*>(a1.devicePointer) - static_cast<const uint8_t*>(a0.devicePointer) !=
        static_cast<ptrdiff_t>(bytes - 1))
        return nullptr;
    return a0.devicePointer;
}

// sdf_render_host with mapped host buffers: one trace over all rays (level 0
// reads orig / dir from host memory), then on one stream the normal mapping
// (writing the hits' normals to host memory) and on another the copy of the
// end points and hit flags.  orig, dir and nrm are device addresses of host
// memory (nrm that of out_normal_host).
int render_mapped(const sdf_trace_params* params, sdf_net_t fine, const float* orig, const float* dir, int64_t n,
                  float* out_pos, uint8_t* out_hit, float* out_normal_host, float* nrm, HostPipe& hp, cudaStream_t s) {
    int dev = -1;
    int rc = validate_trace_params(params, &dev);
    if (rc) return rc;
    if (fine->precision != SDF_FP32 && !tc_grad_supported(fine->width, fine->n_hidden))
        return fail(SDF_ERR_UNSUPPORTED, "tensor-core gradients of a (%d,%d) network are not built", fine->width,
                    fine->n_hidden);
    DeviceInfo di;
    if ((rc = device_info(dev, &di))) return rc;
    const size_t un = static_cast<size_t>(n);
    const size_t ts = (trace_scratch_bytes(params->n_levels, n) + 255) & ~size_t(255);
    const size_t gs = (grad_scratch_bytes(n, true) + 255) & ~size_t(255);
    const size_t fb = (4 * un * sizeof(float) + un + 255) & ~size_t(255);  // pos (3n), t (n), hit (n)
    const size_t zb = 3 * un * sizeof(float);                               // zeros for the normals
    void* block = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&block, ts + gs + fb + zb, di.pool, s);
    if (e != cudaSuccess) return cuda_fail(e, "allocating the frame buffers");
    uint8_t* b = static_cast<uint8_t*>(block);
    float* d_pos = reinterpret_cast<float*>(b + ts + gs);
    float* d_t = d_pos + 3 * un;
    uint8_t* d_hit = reinterpret_cast<uint8_t*>(d_t + un);
    void* d_zero = b + ts + gs + fb;
    cudaStream_t c = hp.cmp[0];
    if ((e = cudaEventRecord(hp.start, s)) == cudaSuccess && (e = cudaStreamWaitEvent(c, hp.start, 0)) == cudaSuccess &&
        (e = cudaStreamWaitEvent(hp.in, hp.start, 0)) == cudaSuccess &&
        (e = cudaStreamWaitEvent(hp.out, hp.start, 0)) == cudaSuccess &&
        // while the rays are traced, the copy engine clears the host normals
        // (the normal mapping then writes the hits' entries only)
        (e = cudaMemsetAsync(d_zero, 0, zb, hp.in)) == cudaSuccess &&
        (e = cudaMemcpyAsync(out_normal_host, d_zero, zb, cudaMemcpyDeviceToHost, hp.in)) == cudaSuccess &&
        (e = cudaEventRecord(hp.ev_cmp[1], hp.in)) == cudaSuccess) {
        rc = launch_levels(params, orig, dir, n, d_pos, d_t, d_hit, nullptr, b, di.d_status, di.num_sms, nullptr, c);
        // then the normals of the hits on c, and the end points and hit flags
        // copied back on `out` meanwhile
        if (rc == SDF_OK && (e = cudaEventRecord(hp.ev_in[0], c)) == cudaSuccess &&
            (e = cudaStreamWaitEvent(hp.out, hp.ev_in[0], 0)) == cudaSuccess &&
            (e = cudaMemcpyAsync(out_pos, d_pos, 3 * un * sizeof(float), cudaMemcpyDeviceToHost, hp.out)) ==
                cudaSuccess &&
            (e = cudaMemcpyAsync(out_hit, d_hit, un, cudaMemcpyDeviceToHost, hp.out)) == cudaSuccess &&
            (e = cudaStreamWaitEvent(c, hp.ev_cmp[1], 0)) == cudaSuccess)
            rc = launch_gradients(fine, d_pos, nullptr, d_hit, n, nrm, 1, b + ts, di.d_status, di.num_sms, c, false);
    }
    cudaError_t e2 = cudaEventRecord(hp.ev_cmp[0], c);
    if (e2 == cudaSuccess) e2 = cudaEventRecord(hp.ev_cmp[1], hp.in);
    if (e2 == cudaSuccess) e2 = cudaEventRecord(hp.done, hp.out);
    if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(s, hp.ev_cmp[0], 0);
    if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(s, hp.ev_cmp[1], 0);
    if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(s, hp.done, 0);
    if (e2 != cudaSuccess) {
        cudaStreamSynchronize(c);
        cudaStreamSynchronize(hp.in);
        cudaStreamSynchronize(hp.out);
    }
    cudaFreeAsync(block, s);
    const cudaError_t e3 = cudaStreamSynchronize(s);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "enqueueing the frame");
    if (e2 != cudaSuccess) return cuda_fail(e2, "ordering the frame's streams");
    if (e3 != cudaSuccess) return cuda_fail(e3, "cudaStreamSynchronize");
    return SDF_OK;
}

// ---------------------------------------------------------------------------
// Frame queues: host frames rendered back to back.  Every slot owns device
// copies of one frame's rays and results and a plan (CUDA graph) over them;
// the rays of frame k + 1 go in and the results of frame k - 1 come out on
// the copy streams while frame k's graph runs.  Consecutive frames run on
// two compute streams, so one frame's trace can start on the SMs the tail of
// the previous frame's trace leaves idle.
// ---------------------------------------------------------------------------
constexpr int kMaxQueueDepth = 4;

struct QueueSlot {
    void* block = nullptr;  // orig, dir, pos, normal (3n floats each), t (n floats), hit (n bytes)
    float *orig = nullptr, *dir = nullptr, *pos = nullptr, *nrm = nullptr, *t = nullptr;
    uint8_t* hit = nullptr;
    sdf_plan_t plan = nullptr;
    cudaEvent_t ev_in = nullptr, ev_cmp = nullptr, ev_out = nullptr;
    int64_t ticket = -1;  // frame in this slot (-1: none yet)
};

}  // namespace

struct sdf_frame_queue {
    int device = 0;
    int depth = 0;
    int64_t n = 0;
    int64_t next = 0;  // ticket of the next frame
    cudaStream_t in = nullptr, cmp[2] = {}, out = nullptr;
    QueueSlot slot[kMaxQueueDepth];
};

namespace {

void free_queue(sdf_frame_queue* q) {
    if (!q) return;
    DeviceGuard g(q->device);
    for (cudaStream_t st : {q->in, q->cmp[0], q->cmp[1], q->out})
        if (st) cudaStreamSynchronize(st);
    for (QueueSlot& sl : q->slot) {
        if (sl.plan) free_plan(sl.plan);
        if (sl.block) cudaFree(sl.block);
        for (cudaEvent_t ev : {sl.ev_in, sl.ev_cmp, sl.ev_out})
            if (ev) cudaEventDestroy(ev);
    }
    for (cudaStream_t st : {q->in, q->cmp[0], q->cmp[1], q->out})
        if (st) cudaStreamDestroy(st);
    delete q;
}

int queue_create(const sdf_trace_params* P, sdf_net_t fine, int64_t n, int depth, sdf_frame_queue_t* out) {
    if (!out) return fail(SDF_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!P) return fail(SDF_ERR_ARG, "params is NULL");
    if (!fine) return fail(SDF_ERR_ARG, "fine is NULL");
    if (n < 1 || n > 0x7fffffffLL) return fail(SDF_ERR_ARG, "n = %lld out of range", static_cast<long long>(n));
    if (depth < 1 || depth > kMaxQueueDepth) return fail(SDF_ERR_ARG, "depth = %d out of range 1..%d", depth, kMaxQueueDepth);
    if (P->ray_time) return fail(SDF_ERR_ARG, "frame queues take no per-ray times");
    int dev = -1;
    int rc = validate_trace_params(P, &dev);
    if (rc) return rc;
    if (fine->device != dev) return fail(SDF_ERR_ARG, "fine network on another device");
    DeviceGuard g(dev);
    if (!g.ok) return fail(SDF_ERR_CUDA, "cudaSetDevice(%d) failed", dev);
    sdf_frame_queue* q = new sdf_frame_queue;
    q->device = dev;
    q->depth = depth;
    q->n = n;
    cudaError_t e = cudaSuccess;
    for (cudaStream_t* st : {&q->in, &q->cmp[0], &q->cmp[1], &q->out})
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(st, cudaStreamNonBlocking);
    const size_t un = static_cast<size_t>(n);
    const size_t f3 = (3 * un * sizeof(float) + 255) & ~size_t(255), f1 = (un * sizeof(float) + 255) & ~size_t(255);
    for (int k = 0; k < depth && e == cudaSuccess && rc == SDF_OK; ++k) {
        QueueSlot& sl = q->slot[k];
        for (cudaEvent_t* ev : {&sl.ev_in, &sl.ev_cmp, &sl.ev_out})
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(&sl.block, 4 * f3 + f1 + un);
        if (e != cudaSuccess) break;
        uint8_t* b = static_cast<uint8_t*>(sl.block);
        sl.orig = reinterpret_cast<float*>(b);
        sl.dir = reinterpret_cast<float*>(b + f3);
        sl.pos = reinterpret_cast<float*>(b + 2 * f3);
        sl.nrm = reinterpret_cast<float*>(b + 3 * f3);
        sl.t = reinterpret_cast<float*>(b + 4 * f3);
        sl.hit = b + 4 * f3 + f1;
        sdf_frame_batch fb{};
        fb.orig = sl.orig;
        fb.dir = sl.dir;
        fb.n = n;
        fb.out_pos = sl.pos;
        fb.out_t = sl.t;
        fb.out_hit = sl.hit;
        fb.out_normal = sl.nrm;
        rc = plan_create(P, fine, &fb, 0, q->cmp[0], &sl.plan);
    }
    if (rc == SDF_OK && e != cudaSuccess) rc = cuda_fail(e, "creating the frame queue");
    if (rc) {
        free_queue(q);
        return rc;
    }
    *out = q;
    return SDF_OK;
}

int queue_submit(sdf_frame_queue* q, const float* orig, const float* dir, float* out_pos, uint8_t* out_hit,
                 float* out_normal, int64_t* ticket) {
    if (!q) return fail(SDF_ERR_ARG, "queue is NULL");
    if (!orig || !dir || !out_pos || !out_hit || !out_normal) return fail(SDF_ERR_ARG, "NULL host buffer");
    DeviceGuard g(q->device);
    if (!g.ok) return fail(SDF_ERR_CUDA, "cudaSetDevice(%d) failed", q->device);
    QueueSlot& sl = q->slot[q->next % q->depth];
    const cudaStream_t cmp = q->cmp[q->next & 1];
    cudaError_t e = cudaSuccess;
    // the slot's previous frame is out of its buffers once its results have left
    if (sl.ticket >= 0 && (e = cudaEventSynchronize(sl.ev_out)) != cudaSuccess)
        return cuda_fail(e, "waiting for the slot's previous frame");
    const size_t b3 = 3 * static_cast<size_t>(q->n) * sizeof(float), b1 = static_cast<size_t>(q->n);
    if ((e = cudaMemcpyAsync(sl.orig, orig, b3, cudaMemcpyHostToDevice, q->in)) != cudaSuccess ||
        (e = cudaMemcpyAsync(sl.dir, dir, b3, cudaMemcpyHostToDevice, q->in)) != cudaSuccess ||
        (e = cudaEventRecord(sl.ev_in, q->in)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(cmp, sl.ev_in, 0)) != cudaSuccess ||
        (e = cudaGraphLaunch(sl.plan->exec, cmp)) != cudaSuccess ||
        (e = cudaEventRecord(sl.ev_cmp, cmp)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(q->out, sl.ev_cmp, 0)) != cudaSuccess ||
        (e = cudaMemcpyAsync(out_pos, sl.pos, b3, cudaMemcpyDeviceToHost, q->out)) != cudaSuccess ||
        (e = cudaMemcpyAsync(out_hit, sl.hit, b1, cudaMemcpyDeviceToHost, q->out)) != cudaSuccess ||
        (e = cudaMemcpyAsync(out_normal, sl.nrm, b3, cudaMemcpyDeviceToHost, q->out)) != cudaSuccess ||
        (e = cudaEventRecord(sl.ev_out, q->out)) != cudaSuccess)
        return cuda_fail(e, "enqueueing the frame");
    sl.ticket = q->next;
    if (ticket) *ticket = q->next;
    ++q->next;
    return SDF_OK;
}

int queue_wait(sdf_frame_queue* q, int64_t ticket) {
    if (!q) return fail(SDF_ERR_ARG, "queue is NULL");
    if (ticket >= q->next) return fail(SDF_ERR_ARG, "frame %lld was not submitted", static_cast<long long>(ticket));
    if (ticket < 0) ticket = q->next - 1;
    if (ticket < 0) return SDF_OK;  // nothing submitted
    DeviceGuard g(q->device);
    if (!g.ok) return fail(SDF_ERR_CUDA, "cudaSetDevice(%d) failed", q->device);
    // the copies out run in frame order on one stream: the event of the frame's
    // slot (or of a later frame that reused it) covers the frame and all before it
    cudaError_t e = cudaEventSynchronize(q->slot[ticket % q->depth].ev_out);
    if (e != cudaSuccess) return cuda_fail(e, "waiting for the frame");
    DeviceInfo di;
    int rc = device_info(q->device, &di);
    if (rc) return rc;
    int status = 0;
    e = cudaMemcpy(&status, di.d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading the status word");
    if (status != 0) {
        const int zero = 0;
        cudaMemcpy(di.d_status, &zero, sizeof(int), cudaMemcpyHostToDevice);
        return fail(status, "device reported status %d (a bounded wait expired)", status);
    }
    return SDF_OK;
}

}  // namespace

extern "C" {

int sdf_net_load_mem(const void* bytes, size_t n_bytes, int precision, int device, sdf_net_t* out) {
    return load_from_memory(static_cast<const uint8_t*>(bytes), n_bytes, precision, device, out);
}

int sdf_net_load(const char* path, int precision, int device, sdf_net_t* out) {
    if (!out) return fail(SDF_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!path) return fail(SDF_ERR_ARG, "path is NULL");
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return fail(SDF_ERR_FILE, "cannot open %s", path);
    std::vector<uint8_t> buf;
    uint8_t tmp[1 << 16];
    size_t got;
    while ((got = std::fread(tmp, 1, sizeof(tmp), fp)) > 0) buf.insert(buf.end(), tmp, tmp + got);
    const bool err = std::ferror(fp) != 0;
    std::fclose(fp);
    if (err) return fail(SDF_ERR_FILE, "error reading %s", path);
    return load_from_memory(buf.data(), buf.size(), precision, device, out);
}

int sdf_net_info(sdf_net_t net, int* in_dim, int* width, int* n_hidden, double* lipschitz) {
    if (!net) return fail(SDF_ERR_ARG, "net is NULL");
    if (in_dim) *in_dim = net->in_dim;
    if (width) *width = net->width;
    if (n_hidden) *n_hidden = net->n_hidden;
    if (lipschitz) *lipschitz = net->lipschitz;
    return SDF_OK;
}

int sdf_net_set_time(sdf_net_t net, float time) {
    if (!net) return fail(SDF_ERR_ARG, "net is NULL");
    if (!std::isfinite(time)) return fail(SDF_ERR_ARG, "time must be finite");
    net->time = time;
    return SDF_OK;
}

void sdf_net_free(sdf_net_t net) { free_net(net); }

int sdf_trace_multiscale(const sdf_trace_params* params, const float* orig, const float* dir, int64_t n,
                         float* out_pos, float* out_t, uint8_t* out_hit, uint16_t* out_iters, void* cuda_stream) {
    return trace_impl(params, orig, dir, n, out_pos, out_t, out_hit, out_iters,
                      static_cast<cudaStream_t>(cuda_stream));
}

int sdf_normals(sdf_net_t net, const float* pts, int64_t n, float* out_grad, void* cuda_stream) {
    return grad_impl(net, pts, nullptr, nullptr, n, out_grad, 0, static_cast<cudaStream_t>(cuda_stream));
}

int sdf_normal_map(sdf_net_t fine, const float* pts, const uint8_t* mask, int64_t n, float* out_normal,
                   void* cuda_stream) {
    return grad_impl(fine, pts, nullptr, mask, n, out_normal, 1, static_cast<cudaStream_t>(cuda_stream));
}

int sdf_normal_map_timed(sdf_net_t fine, const float* pts, const float* pt_time, const uint8_t* mask, int64_t n,
                         float* out_normal, void* cuda_stream) {
    if (!pt_time) return fail(SDF_ERR_ARG, "time is NULL");
    return grad_impl(fine, pts, pt_time, mask, n, out_normal, 1, static_cast<cudaStream_t>(cuda_stream));
}

int sdf_render_host(const sdf_trace_params* params, sdf_net_t fine, const float* orig, const float* dir, int64_t n,
                    float* out_pos, uint8_t* out_hit, float* out_normal, void* cuda_stream) {
    if (!params || !params->nets || params->n_levels < 1 || !params->nets[0])
        return fail(SDF_ERR_ARG, "params / nets missing");
    if (!fine) return fail(SDF_ERR_ARG, "fine is NULL");
    if (!orig || !dir || !out_pos || !out_hit || !out_normal) return fail(SDF_ERR_ARG, "NULL host buffer");
    if (n < 0 || n > 0x7fffffffLL) return fail(SDF_ERR_ARG, "n out of range");
    if (params->ray_time) return fail(SDF_ERR_ARG, "sdf_render_host takes no per-ray times");
    if (n == 0) return SDF_OK;
    const int dev = params->nets[0]->device;
    if (fine->device != dev) return fail(SDF_ERR_ARG, "fine network on another device");
    if (dev < 0 || dev >= 64) return fail(SDF_ERR_ARG, "device %d out of range", dev);
    DeviceGuard g(dev);
    if (!g.ok) return fail(SDF_ERR_CUDA, "cudaSetDevice(%d) failed", dev);
    HostPipe& hp = g_host_pipes[dev];
    std::lock_guard<std::mutex> lock(hp.m);
    int rc = host_pipe_init(&hp);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

    // Page-locked host buffers that the device maps: the kernels read the rays
    // and write the normals over the host link themselves, the copy engine
    // brings back the end points and hit flags while the normals are computed.
    const size_t b3 = 3 * static_cast<size_t>(n) * sizeof(float), b1 = static_cast<size_t>(n);
    const float* m_orig = static_cast<const float*>(mapped_host(orig, b3));
    const float* m_dir = static_cast<const float*>(mapped_host(dir, b3));
    float* m_nrm = static_cast<float*>(const_cast<void*>(mapped_host(out_normal, b3)));
    if (m_orig && m_dir && m_nrm && mapped_host(out_pos, b3) && mapped_host(out_hit, b1))
        return render_mapped(params, fine, m_orig, m_dir, n, out_pos, out_hit, out_normal, m_nrm, hp, s);

    // chunks of rays: the copies of one chunk overlap the kernels of another
    const int nch = n >= (int64_t(1) << 20) ? kHostChunks : (n >= (int64_t(1) << 18) ? 2 : 1);
    const int64_t m = (n + nch - 1) / nch;
    const size_t cm = static_cast<size_t>(m);
    // per chunk: orig, dir, pos, normal (3m floats each), t (m floats), hit (m bytes)
    const size_t chunk_bytes = (13 * cm * sizeof(float) + cm + 255) & ~size_t(255);
    DeviceInfo di;
    if ((rc = device_info(dev, &di))) return rc;
    void* block = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&block, chunk_bytes * nch, di.pool, s);
    if (e != cudaSuccess) return cuda_fail(e, "allocating the frame buffers");
    e = cudaEventRecord(hp.start, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hp.in, hp.start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hp.cmp[0], hp.start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hp.cmp[1], hp.start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hp.out, hp.start, 0);
    for (int c = 0; c < nch && e == cudaSuccess && rc == SDF_OK; ++c) {
        const int64_t lo = c * m, mc = std::min<int64_t>(m, n - lo);
        if (mc <= 0) break;
        const size_t w = static_cast<size_t>(mc) * sizeof(float), hpitch = static_cast<size_t>(n) * sizeof(float);
        uint8_t* b = static_cast<uint8_t*>(block) + c * chunk_bytes;
        float* d_orig = reinterpret_cast<float*>(b);
        float* d_dir = d_orig + 3 * mc;
        float* d_pos = d_dir + 3 * mc;
        float* d_nrm = d_pos + 3 * mc;
        float* d_t = d_nrm + 3 * mc;
        uint8_t* d_hit = reinterpret_cast<uint8_t*>(d_t + mc);
        // rays in (3 rows of mc floats out of the host's (3, n) arrays)
        if ((e = cudaMemcpy2DAsync(d_orig, w, orig + lo, hpitch, w, 3, cudaMemcpyHostToDevice, hp.in)) != cudaSuccess ||
            (e = cudaMemcpy2DAsync(d_dir, w, dir + lo, hpitch, w, 3, cudaMemcpyHostToDevice, hp.in)) != cudaSuccess ||
            (e = cudaEventRecord(hp.ev_in[c], hp.in)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(hp.cmp[c & 1], hp.ev_in[c], 0)) != cudaSuccess)
            break;
        rc = trace_impl(params, d_orig, d_dir, mc, d_pos, d_t, d_hit, nullptr, hp.cmp[c & 1]);
        if (rc == SDF_OK) rc = grad_impl(fine, d_pos, nullptr, d_hit, mc, d_nrm, 1, hp.cmp[c & 1]);
        if (rc) break;
        if ((e = cudaEventRecord(hp.ev_cmp[c], hp.cmp[c & 1])) != cudaSuccess ||
            (e = cudaStreamWaitEvent(hp.out, hp.ev_cmp[c], 0)) != cudaSuccess ||
            (e = cudaMemcpy2DAsync(out_pos + lo, hpitch, d_pos, w, w, 3, cudaMemcpyDeviceToHost, hp.out)) != cudaSuccess ||
            (e = cudaMemcpy2DAsync(out_normal + lo, hpitch, d_nrm, w, w, 3, cudaMemcpyDeviceToHost, hp.out)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(out_hit + lo, d_hit, static_cast<size_t>(mc), cudaMemcpyDeviceToHost, hp.out)) !=
                cudaSuccess)
            break;
    }
    // the caller's stream waits for everything, frees the frame and returns with the results on the host
    cudaError_t e2 = cudaEventRecord(hp.done, hp.out);
    if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(s, hp.done, 0);
    if (e2 != cudaSuccess) {
        cudaStreamSynchronize(hp.in);
        cudaStreamSynchronize(hp.cmp[0]);
        cudaStreamSynchronize(hp.cmp[1]);
        cudaStreamSynchronize(hp.out);
    }
    cudaFreeAsync(block, s);
    const cudaError_t e3 = cudaStreamSynchronize(s);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "enqueueing the frame");
    if (e2 != cudaSuccess) return cuda_fail(e2, "ordering the frame's streams");
    if (e3 != cudaSuccess) return cuda_fail(e3, "cudaStreamSynchronize");
    return SDF_OK;
}

int sdf_sync_status(void* cuda_stream) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    e = cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    DeviceInfo di;
    int rc = device_info(dev, &di);
    if (rc) return rc;
    int status = 0;
    e = cudaMemcpy(&status, di.d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading the status word");
    if (status != 0) {
        const int zero = 0;
        cudaMemcpy(di.d_status, &zero, sizeof(int), cudaMemcpyHostToDevice);
    }
    // the allocation-free entry point latches its kernels' errors in its own array
    int na_status = 0;
    if ((rc = noalloc_take_status(dev, &na_status))) return rc;
    if (status != 0) return fail(status, "device reported status %d (a bounded wait expired)", status);
    if (na_status != 0)
        return fail(na_status, "device reported status %d in sdf_trace_multiscale_noalloc (a bounded wait expired)",
                    na_status);
    return SDF_OK;
}

int sdf_trace_multiscale_noalloc(const sdf_trace_params* P, const float* orig, const float* dir, int64_t n,
                                 float* out_pos, float* out_t, uint8_t* out_hit, uint16_t* out_iters,
                                 void* cuda_stream) {
    // Same contract as sdf_trace_multiscale, with the scratch taken from the
    // static array above instead of the stream-ordered allocator.
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (n > kNoAllocMaxRays)
        return fail(SDF_ERR_ARG, "n = %lld: sdf_trace_multiscale_noalloc handles at most %lld rays per call",
                    static_cast<long long>(n), static_cast<long long>(kNoAllocMaxRays));
    int dev = -1;
    int rc = validate_trace(P, orig, dir, n, out_pos, out_t, out_hit, out_iters, &dev);
    if (rc || n == 0) return rc;
    DeviceGuard g(dev);
    if (!g.ok) return fail(SDF_ERR_CUDA, "cudaSetDevice(%d) failed", dev);
    NoAllocDevice nd;
    if ((rc = noalloc_setup(dev, &nd))) return rc;
    return launch_levels_at(P, orig, dir, n, out_pos, out_t, out_hit, out_iters, nd.scratch->counters,
                            nd.scratch->lists[0], nd.scratch->lists[1], &nd.scratch->status, nd.num_sms, nullptr, s);
}

int sdf_plan_create(const sdf_trace_params* params, sdf_net_t fine, const sdf_frame_batch* batch, int autotune,
                    void* cuda_stream, sdf_plan_t* out) {
    return plan_create(params, fine, batch, autotune, static_cast<cudaStream_t>(cuda_stream), out);
}

int sdf_plan_launch(sdf_plan_t plan, void* cuda_stream) {
    if (!plan) return fail(SDF_ERR_ARG, "plan is NULL");
    if (!plan->exec) return SDF_OK;  // empty batch
    DeviceGuard g(plan->device);
    if (!g.ok) return fail(SDF_ERR_CUDA, "cudaSetDevice(%d) failed", plan->device);
    cudaError_t e = cudaGraphLaunch(plan->exec, static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return SDF_OK;
}

int sdf_plan_info(sdf_plan_t plan, int* tiles, int max_levels, int64_t* n_graph_nodes) {
    if (!plan) return fail(SDF_ERR_ARG, "plan is NULL");
    if (tiles) {
        if (max_levels < plan->n_levels) return fail(SDF_ERR_ARG, "tiles needs %d entries", plan->n_levels);
        for (int j = 0; j < plan->n_levels; ++j) tiles[j] = plan->tiles[j];
    }
    if (n_graph_nodes) *n_graph_nodes = static_cast<int64_t>(plan->n_nodes);
    return SDF_OK;
}

void sdf_plan_free(sdf_plan_t plan) { free_plan(plan); }

int sdf_frame_queue_create(const sdf_trace_params* params, sdf_net_t fine, int64_t n, int depth,
                           sdf_frame_queue_t* queue) {
    return queue_create(params, fine, n, depth, queue);
}

int sdf_frame_queue_submit(sdf_frame_queue_t queue, const float* orig, const float* dir, float* out_pos,
                           uint8_t* out_hit, float* out_normal, int64_t* ticket) {
    return queue_submit(queue, orig, dir, out_pos, out_hit, out_normal, ticket);
}

int sdf_frame_queue_wait(sdf_frame_queue_t queue, int64_t ticket) { return queue_wait(queue, ticket); }

void sdf_frame_queue_free(sdf_frame_queue_t queue) { free_queue(queue); }

// ---------------------------------------------------------------------------
// training path
// ---------------------------------------------------------------------------
static int train_check_precision(int precision) {
    if (precision != SDF_FP32 && precision != SDF_BF16 && precision != SDF_FP16)
        return fail(precision == SDF_FP8 ? SDF_ERR_UNSUPPORTED : SDF_ERR_ARG,
                    "training precision %d: SDF_FP32, SDF_BF16 or SDF_FP16", precision);
    return SDF_OK;
}

static int train_check_shape(int in_dim, int width, int n_hidden) {
    if ((in_dim != 3 && in_dim != 4) || (width != 64 && width != 128 && width != 256) || n_hidden < 1 ||
        n_hidden > kMaxHidden)
        return fail(SDF_ERR_UNSUPPORTED, "training shape in=%d (w=%d, k=%d) not supported (in 3|4, w 64|128|256, "
                                         "1<=k<=%d)",
                    in_dim, width, n_hidden, kMaxHidden);
    return SDF_OK;
}

// Device of a device pointer (SDF_ERR_ARG if it is not one).
static int device_of(const void* p, const char* name, int* dev) {
    if (!p) return fail(SDF_ERR_ARG, "%s is NULL", name);
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return fail(SDF_ERR_ARG, "%s: not a CUDA pointer", name);
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return fail(SDF_ERR_ARG, "%s must be device memory", name);
    *dev = at.device;
    return SDF_OK;
}

int sdf_train_shape_info(int precision, int in_dim, int width, int n_hidden, int64_t n, int64_t* param_count,
                         int64_t* workspace_bytes) {
    int rc = train_check_precision(precision);
    if (rc || (rc = train_check_shape(in_dim, width, n_hidden))) return rc;
    if (n < 0 || n > 0x7fffffffLL) return fail(SDF_ERR_ARG, "n = %lld out of range", static_cast<long long>(n));
    const TrainShape sh = train_shape(in_dim, width, n_hidden);
    if (param_count) *param_count = sh.count;
    if (workspace_bytes)
        *workspace_bytes = static_cast<int64_t>(precision == SDF_FP32 ? train_workspace_bytes(sh, n)
                                                                      : train_tc_workspace_bytes(sh, n));
    return SDF_OK;
}

static int train_prepare(int precision, int in_dim, int width, int n_hidden, const float* theta, const float* pts,
                         const float* pt_time, int64_t n, void* workspace, TrainArgs* a, int* dev) {
    int rc = train_check_precision(precision);
    if (rc || (rc = train_check_shape(in_dim, width, n_hidden))) return rc;
    if (n < 0 || n > 0x7fffffffLL) return fail(SDF_ERR_ARG, "n = %lld out of range", static_cast<long long>(n));
    if (pt_time && in_dim != 4) return fail(SDF_ERR_ARG, "per-point times given for a 3-input network");
    if ((rc = device_of(theta, "theta", dev))) return rc;
    if (reinterpret_cast<uintptr_t>(theta) % 16) return fail(SDF_ERR_ARG, "theta must be 16-byte aligned");
    if (n > 0) {
        if ((rc = check_device_ptr(pts, *dev, "pts")) || (rc = check_device_ptr(workspace, *dev, "workspace")))
            return rc;
        if (reinterpret_cast<uintptr_t>(workspace) % 256) return fail(SDF_ERR_ARG, "workspace must be 256-byte aligned");
        if (pt_time && (rc = check_device_ptr(pt_time, *dev, "time"))) return rc;
    }
    *a = TrainArgs{};
    a->sh = train_shape(in_dim, width, n_hidden);
    a->theta = theta;
    a->pts = pts;
    a->pt_time = pt_time;
    a->n = n;
    a->w = precision == SDF_FP32 ? train_work(a->sh, n, workspace) : train_tc_work(a->sh, n, workspace);
    return SDF_OK;
}

int sdf_train_forward(int precision, int in_dim, int width, int n_hidden, const float* theta, const float* pts,
                      const float* pt_time, int64_t n, float* out_f, float* out_grad, void* workspace,
                      void* cuda_stream) {
    TrainArgs a;
    int dev = -1;
    int rc = train_prepare(precision, in_dim, width, n_hidden, theta, pts, pt_time, n, workspace, &a, &dev);
    if (rc || n == 0) return rc;
    if ((rc = check_device_ptr(out_f, dev, "out_f")) || (rc = check_device_ptr(out_grad, dev, "out_grad"))) return rc;
    DeviceGuard g(dev);
    if (!g.ok) return fail(SDF_ERR_CUDA, "cudaSetDevice(%d) failed", dev);
    DeviceInfo di;
    if ((rc = device_info(dev, &di))) return rc;
    a.out_f = out_f;
    a.out_grad = out_grad;
    a.status = di.d_status;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = precision == SDF_FP32 ? launch_train_forward(a, di.num_sms, s)
                                          : launch_train_forward_tc(a, precision == SDF_FP16, di.num_sms, s);
    if (e != cudaSuccess) return cuda_fail(e, "launching the training forward");
    return SDF_OK;
}

int sdf_train_backward(int precision, int in_dim, int width, int n_hidden, const float* theta, const float* pts,
                       const float* pt_time, int64_t n, const float* d_f, const float* d_grad, void* workspace,
                       float* d_theta, void* cuda_stream) {
    TrainArgs a;
    int dev = -1;
    int rc = train_prepare(precision, in_dim, width, n_hidden, theta, pts, pt_time, n, workspace, &a, &dev);
    if (rc || n == 0) return rc;
    if ((rc = check_device_ptr(d_f, dev, "d_f")) || (rc = check_device_ptr(d_grad, dev, "d_grad")) ||
        (rc = check_device_ptr(d_theta, dev, "d_theta")))
        return rc;
    if (reinterpret_cast<uintptr_t>(d_theta) % 16) return fail(SDF_ERR_ARG, "d_theta must be 16-byte aligned");
    DeviceGuard g(dev);
    if (!g.ok) return fail(SDF_ERR_CUDA, "cudaSetDevice(%d) failed", dev);
    DeviceInfo di;
    if ((rc = device_info(dev, &di))) return rc;
    a.d_f = d_f;
    a.d_grad = d_grad;
    a.d_theta = d_theta;
    a.status = di.d_status;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = precision == SDF_FP32 ? launch_train_backward(a, di.num_sms, s)
                                          : launch_train_backward_tc(a, precision == SDF_FP16, di.num_sms, s);
    if (e != cudaSuccess) return cuda_fail(e, "launching the training backward");
    return SDF_OK;
}

int sdf_fit_loss(const float* f, const float* grad, const float* target_f, const float* target_grad,
                 const uint8_t* near, int64_t n, float lam_n, float lam_e, float* d_f, float* d_grad, double* loss,
                 void* cuda_stream) {
    if (n < 0 || n > 0x7fffffffLL) return fail(SDF_ERR_ARG, "n = %lld out of range", static_cast<long long>(n));
    if (!std::isfinite(lam_n) || !std::isfinite(lam_e)) return fail(SDF_ERR_ARG, "weights must be finite");
    if (n == 0) return SDF_OK;
    int dev = -1, rc;
    if ((rc = device_of(f, "f", &dev))) return rc;
    if ((rc = check_device_ptr(grad, dev, "grad")) || (rc = check_device_ptr(target_f, dev, "target_f")) ||
        (rc = check_device_ptr(target_grad, dev, "target_grad")) || (rc = check_device_ptr(near, dev, "near")) ||
        (rc = check_device_ptr(d_f, dev, "d_f")) || (rc = check_device_ptr(d_grad, dev, "d_grad")) ||
        (rc = check_device_ptr(loss, dev, "loss")))
        return rc;
    DeviceGuard g(dev);
    if (!g.ok) return fail(SDF_ERR_CUDA, "cudaSetDevice(%d) failed", dev);
    DeviceInfo di;
    if ((rc = device_info(dev, &di))) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    Scratch sc;
    sc.s = s;
    cudaError_t e = cudaMallocFromPoolAsync(&sc.ptr, 64, di.pool, s);
    if (e != cudaSuccess) return cuda_fail(e, "allocating scratch");
    double* sums = static_cast<double*>(sc.ptr);
    auto* cnt = reinterpret_cast<unsigned long long*>(sums + 4);
    e = launch_fit_loss(f, grad, target_f, target_grad, near, n, lam_n, lam_e, d_f, d_grad, sums, cnt, loss, di.num_sms,
                        s);
    if (e != cudaSuccess) return cuda_fail(e, "launching the fitting objective");
    return SDF_OK;
}

int sdf_adam_step(float* theta, const float* grad, float* m, float* v, int64_t count, float lr, float beta1,
                  float beta2, float eps, int step, void* cuda_stream) {
    if (count < 0) return fail(SDF_ERR_ARG, "count < 0");
    if (step < 1) return fail(SDF_ERR_ARG, "step counts from 1");
    if (!(beta1 >= 0.0f && beta1 < 1.0f && beta2 >= 0.0f && beta2 < 1.0f) || !std::isfinite(lr) || !(eps > 0.0f))
        return fail(SDF_ERR_ARG, "bad Adam hyper-parameters");
    if (count == 0) return SDF_OK;
    int dev = -1, rc;
    if ((rc = device_of(theta, "theta", &dev))) return rc;
    if ((rc = check_device_ptr(grad, dev, "grad")) || (rc = check_device_ptr(m, dev, "m")) ||
        (rc = check_device_ptr(v, dev, "v")))
        return rc;
    DeviceGuard g(dev);
    if (!g.ok) return fail(SDF_ERR_CUDA, "cudaSetDevice(%d) failed", dev);
    DeviceInfo di;
    if ((rc = device_info(dev, &di))) return rc;
    cudaError_t e = launch_adam(theta, grad, m, v, count, lr, beta1, beta2, eps, step, di.num_sms,
                                static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return cuda_fail(e, "launching Adam");
    return SDF_OK;
}

int sdf_selftest_wait_timeout(int device, int64_t budget_us, void* cuda_stream) {
    if (budget_us < 1 || budget_us > 10000000) return fail(SDF_ERR_ARG, "budget_us out of range 1..1e7");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return fail(SDF_ERR_ARG, "device %d not available", device);
    }
    DeviceGuard g(device);
    if (!g.ok) return fail(SDF_ERR_CUDA, "cudaSetDevice(%d) failed", device);
    DeviceInfo di;
    int rc = device_info(device, &di);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // the status word must be clear before, and must read the timeout after
    rc = sdf_sync_status(cuda_stream);
    if (rc) return rc;
    cudaError_t e = launch_wait_timeout_selftest(di.d_status, static_cast<unsigned long long>(budget_us) * 1000ull, s);
    if (e != cudaSuccess) return cuda_fail(e, "launching the timeout self-test");
    rc = sdf_sync_status(cuda_stream);
    if (rc == SDF_ERR_TIMEOUT) return SDF_OK;
    return rc ? rc : fail(SDF_ERR_CUDA, "the bounded wait did not report its expiry");
}

int sdf_selftest_noalloc_timeout(int device, int64_t budget_us, void* cuda_stream) {
    if (budget_us < 1 || budget_us > 10000000) return fail(SDF_ERR_ARG, "budget_us out of range 1..1e7");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return fail(SDF_ERR_ARG, "device %d not available", device);
    }
    DeviceGuard g(device);
    if (!g.ok) return fail(SDF_ERR_CUDA, "cudaSetDevice(%d) failed", device);
    NoAllocDevice nd;
    int rc = noalloc_setup(device, &nd);
    if (rc) return rc;
    rc = sdf_sync_status(cuda_stream);
    if (rc) return rc;
    cudaError_t e = launch_wait_timeout_selftest(&nd.scratch->status,
                                                 static_cast<unsigned long long>(budget_us) * 1000ull,
                                                 static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return cuda_fail(e, "launching the timeout self-test");
    rc = sdf_sync_status(cuda_stream);
    if (rc == SDF_ERR_TIMEOUT) return SDF_OK;
    return rc ? rc : fail(SDF_ERR_CUDA, "the expiry latched in the static scratch was not reported");
}

int sdf_theta_from_image(const void* bytes, size_t n_bytes, float* theta, int64_t capacity, int64_t* count,
                         int* in_dim, int* width, int* n_hidden) {
    ParsedImage img;
    int rc = parse_image(static_cast<const uint8_t*>(bytes), n_bytes, &img);
    if (rc) return rc;
    const int64_t W = img.W, IN = img.IN, KH = img.KH;
    const int64_t total = W * IN + W + KH * (W * W + W) + W + 1;
    if (count) *count = total;
    if (in_dim) *in_dim = img.IN;
    if (width) *width = img.W;
    if (n_hidden) *n_hidden = img.KH;
    if (!theta) return SDF_OK;
    if (capacity < total)
        return fail(SDF_ERR_ARG, "theta holds %lld floats, the image has %lld parameters",
                    static_cast<long long>(capacity), static_cast<long long>(total));
    int64_t o = 0;
    for (int l = 0; l <= img.KH; ++l) {
        for (double v : img.Wl[l]) theta[o++] = static_cast<float>(v);
        for (double v : img.bl[l]) theta[o++] = static_cast<float>(v);
    }
    for (double v : img.wout) theta[o++] = static_cast<float>(v);
    theta[o++] = img.bout;
    return SDF_OK;
}

int sdf_eval_sine(int variant, const float* x, int64_t n, float* out_sin, float* out_cos, void* cuda_stream) {
    if (variant != 0 && variant != 1) return fail(SDF_ERR_ARG, "variant must be 0 (FP32 path) or 1 (tensor-core paths)");
    if (n < 0) return fail(SDF_ERR_ARG, "n < 0");
    if (n == 0) return SDF_OK;
    int dev = -1, rc;
    if ((rc = device_of(x, "x", &dev))) return rc;
    if ((rc = check_device_ptr(out_sin, dev, "out_sin")) || (rc = check_device_ptr(out_cos, dev, "out_cos"))) return rc;
    DeviceGuard g(dev);
    if (!g.ok) return fail(SDF_ERR_CUDA, "cudaSetDevice(%d) failed", dev);
    DeviceInfo di;
    if ((rc = device_info(dev, &di))) return rc;
    cudaError_t e = launch_sine_eval(variant, x, n, out_sin, out_cos, di.num_sms, static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return cuda_fail(e, "launching the sine evaluation");
    return SDF_OK;
}

int sdf_measure_sine_rate(int device, double* sines_per_s, void* cuda_stream) {
    if (!sines_per_s) return fail(SDF_ERR_ARG, "sines_per_s is NULL");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return fail(SDF_ERR_ARG, "device %d not available", device);
    }
    DeviceGuard g(device);
    if (!g.ok) return fail(SDF_ERR_CUDA, "cudaSetDevice(%d) failed", device);
    DeviceInfo di;
    int rc = device_info(device, &di);
    if (rc) return rc;
    cudaError_t e = measure_sine_rate(di.num_sms, static_cast<cudaStream_t>(cuda_stream), sines_per_s);
    if (e != cudaSuccess) return cuda_fail(e, "measuring the sine rate");
    return SDF_OK;
}

const char* sdf_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
