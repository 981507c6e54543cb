// Checks builds (-DCDF_CHECKS): offset checks of the step kernels and canary
// pads around device buffers.  In a normal build this file holds only the
// pass-through allocation calls and the two C entry points, which report that
// the checks are not built in.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "../../include/cdf_lb.h"
#include "lb_device.cuh"
#include "lb_internal.h"

namespace cdflb {

#ifdef CDF_CHECKS

namespace {

constexpr size_t kPad = 64 * 1024;  // bytes of pattern before and after each buffer (keeps 256-byte alignment)
constexpr unsigned char kCanary = 0xA5;
constexpr int kMaxDevices = 64;

std::mutex g_mu;
std::unordered_map<void *, size_t> g_live;  // user pointer -> requested bytes
unsigned long long *g_word[kMaxDevices] = {};

char *base_of(void *p) { return static_cast<char *>(p) - kPad; }

// One pad: kPad bytes at `pad`; returns the first byte that lost the pattern or -1.
long long damaged_byte(const char *pad, std::vector<unsigned char> &host) {
    if (cudaMemcpy(host.data(), pad, kPad, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return -2;
    }
    for (size_t i = 0; i < kPad; ++i)
        if (host[i] != kCanary) return (long long)i;
    return -1;
}

// Offset probe of the self-test: offsets 64..95 of a 64-float buffer go
// through the check, which turns them into 0.
__global__ void checks_probe_kernel(float *buf, unsigned long long *word) {
    LbParams p{};
    p.check = word;
    const int off = 64 + (int)threadIdx.x;
    const int k = CDF_CHK(p, off, 64, 99);
    buf[k] = buf[k] + 0.f;
}

}  // namespace

unsigned long long *check_word() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_word[dev]) {
        void *p = nullptr;
        if (cudaMalloc(&p, sizeof(unsigned long long)) != cudaSuccess ||
            cudaMemset(p, 0, sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_word[dev] = static_cast<unsigned long long *>(p);
    }
    return g_word[dev];
}

cudaError_t dev_alloc(void **p, size_t bytes) {
    *p = nullptr;
    char *base = nullptr;
    cudaError_t e = cudaMalloc((void **)&base, bytes + 2 * kPad);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemset(base, kCanary, kPad)) != cudaSuccess ||
        (e = cudaMemset(base + kPad + bytes, kCanary, kPad)) != cudaSuccess ||
        (e = cudaDeviceSynchronize()) != cudaSuccess) {
        cudaFree(base);
        return e;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    g_live[base + kPad] = bytes;
    *p = base + kPad;
    return cudaSuccess;
}

void dev_free(void *p) {
    if (!p) return;
    bool padded;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        padded = g_live.erase(p) == 1;
    }
    cudaFree(padded ? base_of(p) : p);  // a buffer that dev_alloc did not make has no pads
}

cdf_status checks_verify(cudaStream_t s) {
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        const cudaError_t e = cudaGetLastError();
        char msg[200];
        std::snprintf(msg, sizeof msg, "checks: stream synchronize failed: %s", cudaGetErrorString(e));
        return report_error(CDF_ECUDA, msg);
    }
    unsigned long long *w = check_word();
    unsigned long long v = 0;
    if (w && cudaMemcpy(&v, w, sizeof v, cudaMemcpyDeviceToHost) == cudaSuccess && v) {
        cudaMemset(w, 0, sizeof v);
        cudaDeviceSynchronize();
        const int site = (int)((v >> 48) & 0x7fff);
        long long off = (long long)(v & 0xffffffffffffull);
        if (off & (1ll << 47)) off -= (1ll << 48);  // 48-bit two's complement
        char msg[200];
        std::snprintf(msg, sizeof msg, "checks: out-of-range offset %lld at access site %d", off, site);
        return report_error(CDF_ECHECK, msg);
    }
    std::vector<unsigned char> host(kPad);
    std::lock_guard<std::mutex> lock(g_mu);
    for (const auto &kv : g_live) {
        char *user = static_cast<char *>(kv.first);
        const size_t bytes = kv.second;
        for (int side = 0; side < 2; ++side) {
            char *pad = side == 0 ? base_of(user) : user + bytes;
            const long long b = damaged_byte(pad, host);
            if (b == -1) continue;
            cudaMemset(pad, kCanary, kPad);  // restore for the calls that follow
            cudaDeviceSynchronize();
            char msg[200];
            std::snprintf(msg, sizeof msg, "checks: canary pad %s a buffer of %zu bytes damaged at pad byte %lld",
                          side == 0 ? "before" : "after", bytes, b);
            return report_error(CDF_ECHECK, msg);
        }
    }
    return CDF_OK;
}

#else  // normal build

unsigned long long *check_word() { return nullptr; }
cudaError_t dev_alloc(void **p, size_t bytes) { return cudaMalloc(p, bytes); }
void dev_free(void *p) { cudaFree(p); }

#endif

}  // namespace cdflb

extern "C" {

int cdf_checks_enabled(void) {
#ifdef CDF_CHECKS
    return 1;
#else
    return 0;
#endif
}

cdf_status cdf_checks_selftest(int which) {
#ifdef CDF_CHECKS
    using namespace cdflb;
    if (which != 0 && which != 1) return report_error(CDF_EINVAL, "which must be 0 or 1");
    if (which == 0) {
        float *buf = nullptr;
        if (dev_alloc((void **)&buf, 64 * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return report_error(CDF_ENOMEM, "checks self-test: allocation failed");
        }
        cudaMemset(buf, 0, 64 * sizeof(float));
        checks_probe_kernel<<<1, 32>>>(buf, check_word());
        cudaError_t e = cudaGetLastError();
        cdf_status st = e == cudaSuccess ? checks_verify(nullptr) : report_error(CDF_ECUDA, cudaGetErrorString(e));
        dev_free(buf);
        return st;
    }
    char *buf = nullptr;
    if (dev_alloc((void **)&buf, 256) != cudaSuccess) {
        cudaGetLastError();
        return report_error(CDF_ENOMEM, "checks self-test: allocation failed");
    }
    // byte 5 of the pad behind the buffer: inside the allocation, outside the buffer
    cudaMemset(buf + 256 + 5, 0, 1);
    cdf_status st = checks_verify(nullptr);
    dev_free(buf);
    return st;
#else
    (void)which;
    return cdflb::report_error(CDF_EINVAL, "not a checks build (build with -DCDF_CHECKS)");
#endif
}

}  // extern "C"
