// Inference of the warm-start network without any allocation (kamino_mlp_predict_static).
//
// kamino_mlp_predict runs the network with the activation workspace its kamino_mlp_t allocated.
// Some callers cannot have memory allocated on their behalf: code that runs while another
// component owns the device allocator (and would see an unexpected cudaMalloc as a leak or a
// synchronisation point), real-time control loops whose latency budget forbids the implicit
// device synchronisation of cudaMalloc / cudaFree, and hosts that pre-plan every byte of device
// memory.  For them this entry point takes its activations from one file-scope device array of
// fixed size, kMaxBytes, which every GPU that loads the library holds until the process exits.
//
// The array's name is only a host-side stand-in in host code: its device address is fetched once
// per device with cudaGetSymbolAddress (the first call on a device does this, so make that first
// call before any stream capture) and passed to the kernels.  The address is cached per device
// ordinal for the life of the process: a cudaDeviceReset destroys the context that holds the array,
// so a process that resets a device must not call this entry point on that device afterwards.  The
// call runs on the calling thread's current device, which must be the one that holds the network
// (the device current at kamino_mlp_create).  All calls share the array, so calls that overlap on
// the GPU (different streams, or several host threads on the same device) race on it; serialise
// them.  Nothing in it needs clearing between calls: every word a call reads was written earlier
// by the same call.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "kamino.h"
#include "kamino_internal.h"
#include "kamino_mlp.h"

namespace {

constexpr size_t kMaxBytes = KAMINO_MLP_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kMaxBytes];

std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {nullptr};

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

// Bytes of the activations of `batch` rows: normalised input (BF16), two ping-pong hidden
// activations (BF16), output (FP32), each 256-byte aligned.
size_t scratch_bytes(size_t batch, size_t din, size_t hidden, size_t dout) {
    return round256(batch * din * 2) + 2 * round256(batch * hidden * 2) + round256(batch * dout * 4);
}

// The largest batch whose activations fit the array (0 if not even one row does).
size_t max_rows(size_t din, size_t hidden, size_t dout) {
    const size_t per = 2 * din + 4 * hidden + 4 * dout;
    size_t b = kMaxBytes > 4 * 256 ? (kMaxBytes - 4 * 256) / per : 0;   // rounding adds < 4 x 256 bytes
    while (scratch_bytes(b + 1, din, hidden, dout) <= kMaxBytes) ++b;
    return b;
}

}  // namespace

extern "C" kamino_status kamino_mlp_predict_static(kamino_mlp_t net, const float *x_dev, int32_t batch,
                                                  float *y_dev, void *stream) {
    using namespace kamino::mlp;
    NetView v;
    if (!net || !x_dev || !y_dev || !net_view(net, &v))
        return kamino::report_error(KAMINO_E_INVALID_ARG, "mlp, x and y must not be NULL");
    if (batch < 1) return kamino::report_error(KAMINO_E_INVALID_ARG, "batch must be >= 1");
    // layout: normalised input (BF16), two ping-pong hidden activations (BF16), output (FP32)
    const size_t bx = round256((size_t)batch * v.din * sizeof(__nv_bfloat16));
    const size_t bh = round256((size_t)batch * v.hidden * sizeof(__nv_bfloat16));
    const size_t need = scratch_bytes((size_t)batch, v.din, v.hidden, v.dout);
    if (need > kMaxBytes) {
        char msg[256];
        snprintf(msg, sizeof(msg),
                 "batch %d needs %zu bytes of static scratch, the library holds %zu (at most %zu rows for this "
                 "network)", batch, need, kMaxBytes, max_rows(v.din, v.hidden, v.dout));
        return kamino::report_error(KAMINO_E_UNSUPPORTED, msg);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return kamino::report_error(KAMINO_E_CUDA, cudaGetErrorString(e));
    if (dev != v.device) {
        char msg[160];
        snprintf(msg, sizeof(msg), "the current device is %d but the network lives on device %d", dev, v.device);
        return kamino::report_error(KAMINO_E_INVALID_ARG, msg);
    }
    if (dev < 0 || dev >= kMaxDevices) return kamino::report_error(KAMINO_E_UNSUPPORTED, "device ordinal too large");
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess || !p)
                return kamino::report_error(KAMINO_E_CUDA, e != cudaSuccess ? cudaGetErrorString(e)
                                                                            : "no device address for the scratch");
            g_scratch_addr[dev] = p;
        }
        base = static_cast<unsigned char *>(g_scratch_addr[dev]);
    }
    __nv_bfloat16 *Xb = reinterpret_cast<__nv_bfloat16 *>(base);
    __nv_bfloat16 *H[2] = {reinterpret_cast<__nv_bfloat16 *>(base + bx),
                           reinterpret_cast<__nv_bfloat16 *>(base + bx + bh)};
    float *Y = reinterpret_cast<float *>(base + bx + 2 * bh);
    cudaStream_t s = (cudaStream_t)stream;
    e = normalize_rows(x_dev, v.din, nullptr, batch, v.xmean, v.xinv, Xb, s);
    const __nv_bfloat16 *in = Xb;
    int din = v.din;
    for (int l = 0; l <= v.layers && e == cudaSuccess; ++l) {
        const bool last = l == v.layers;
        GemmArgs g{};
        g.M = batch;
        g.N = last ? v.dout : v.hidden;
        g.K = din;
        g.A = in; g.sam = din; g.sak = 1;
        g.B = v.PB + v.woff[l]; g.sbk = 1; g.sbn = din;
        g.bias = v.P + v.boff[l];
        if (!last) {
            g.epi = EPI_BIAS_GELU;
            g.Cf = nullptr;
            g.Cb = H[l & 1]; g.ldcb = v.hidden;
            in = H[l & 1];
            din = v.hidden;
        } else {
            g.epi = EPI_BIAS_F32;
            g.Cf = Y; g.ldcf = v.dout;
        }
        e = gemm(g, s);
    }
    if (e == cudaSuccess) e = denormalize(Y, batch, v.dout, v.ymean, v.yinv, y_dev, s);
    if (e != cudaSuccess) return kamino::report_error(KAMINO_E_CUDA, cudaGetErrorString(e));
    return KAMINO_OK;
}
