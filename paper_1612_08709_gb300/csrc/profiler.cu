// Kernel launch counting and optional per-kernel CUDA-event timing.
//
// Every launch made by the library goes through a ProfScope: it always
// increments the launch counter, and when profiling is enabled it records
// a CUDA event pair around the launch on the launch's own stream.  The
// report (tssvd_profile_report) synchronises the device, sums the elapsed
// times per kernel name and releases the events.
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace tssvd {

namespace {

struct Rec {
    const char *name;
    cudaEvent_t a, b;
};

std::atomic<long long> g_launches{0};
std::atomic<int> g_enabled{0};
std::mutex g_mu;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
std::vector<std::pair<const char *, double>> g_host_recs;  // times taken elsewhere

cudaEvent_t take_event()
{
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

}  // namespace

ProfScope::ProfScope(const char *name, cudaStream_t s) : idx(-1), s(s)
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!g_enabled.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lk(g_mu);
    Rec r{name, take_event(), take_event()};
    if (!r.a || !r.b) return;
    if (cudaEventRecord(r.a, s) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    idx = (int)g_recs.size();
    g_recs.push_back(r);
}

ProfScope::~ProfScope()
{
    if (idx < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (idx < (int)g_recs.size()) {
        if (cudaEventRecord(g_recs[idx].b, s) != cudaSuccess) cudaGetLastError();
    }
}

void add_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

bool profiling() { return g_enabled.load(std::memory_order_relaxed) != 0; }

void prof_add_ms(const char *name, double ms)
{
    if (!profiling()) return;
    std::lock_guard<std::mutex> lk(g_mu);
    g_host_recs.emplace_back(name, ms);
}

namespace {

// FP64 fused multiply-add throughput: every thread runs eight independent
// FMA chains (no memory traffic); the sum is stored only when it takes an
// impossible value, so the chains are kept without a store per thread.
__device__ double g_dfma_sink;

__global__ void __launch_bounds__(256) dfma_rate_kernel(int iters, double a, double b)
{
    double x[8];
#pragma unroll
    for (int u = 0; u < 8; u++) x[u] = (double)(threadIdx.x + u);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int r = 0; r < 8; r++) {
#pragma unroll
            for (int u = 0; u < 8; u++) x[u] = fma(x[u], a, b);
        }
    }
    double t = 0.0;
#pragma unroll
    for (int u = 0; u < 8; u++) t += x[u];
    if (t == -1.0) g_dfma_sink = t;
}

}  // namespace

}  // namespace tssvd

using namespace tssvd;

extern "C" {

int tssvd_profile_enable(int on)
{
    int prev = g_enabled.exchange(on ? 1 : 0);
    return prev;
}

long long tssvd_launch_count(void) { return g_launches.load(); }

int tssvd_fp64_fma_rate(double *tflops, void *stream)
{
    if (!tflops) return -1;
    cudaStream_t s = (cudaStream_t)stream;
    // about 0.3 s per run at GB300's rate: long enough for the clocks to
    // leave their idle state in the warm-up run
    const int blocks = num_sms() * 8, threads = 256, iters = 10000;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return TSSVD_ECUDA;
    }
    float best = 0.f;
    int rc = TSSVD_OK;
    for (int r = 0; r < 5 && rc == TSSVD_OK; r++) {
        float ms = 0.f;
        if (cudaEventRecord(e0, s) != cudaSuccess) rc = TSSVD_ECUDA;
        dfma_rate_kernel<<<blocks, threads, 0, s>>>(iters, 0.9999999, 1e-9);
        if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            rc = TSSVD_ECUDA;
        g_launches.fetch_add(1, std::memory_order_relaxed);
        if (rc == TSSVD_OK && r > 0 && (best == 0.f || ms < best)) best = ms;  // first run warms up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != TSSVD_OK || best <= 0.f) {
        cudaGetLastError();
        return TSSVD_ECUDA;
    }
    const double flops = 2.0 * 64.0 * iters * (double)blocks * threads;
    *tflops = flops / (best * 1e-3) / 1e12;
    return TSSVD_OK;
}

size_t tssvd_profile_report(char *buf, size_t len)
{
    std::lock_guard<std::mutex> lk(g_mu);
    cudaDeviceSynchronize();
    const bool consume = (buf != nullptr);
    std::map<std::string, std::pair<long long, double>> agg;
    for (Rec &r : g_recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
            cudaGetLastError();
            ms = 0.f;
        }
        auto &e = agg[r.name];
        e.first += 1;
        e.second += ms;
        if (consume) {
            g_pool.push_back(r.a);
            g_pool.push_back(r.b);
        }
    }
    if (consume) g_recs.clear();
    for (auto &hr : g_host_recs) {
        auto &e = agg[hr.first];
        e.first += 1;
        e.second += hr.second;
    }
    if (consume) g_host_recs.clear();
    std::string out;
    char line[256];
    for (auto &kv : agg) {
        snprintf(line, sizeof(line), "%s %lld %.6f\n", kv.first.c_str(), kv.second.first,
                 kv.second.second);
        out += line;
    }
    if (buf && len > 0) {
        size_t n = out.size() < len - 1 ? out.size() : len - 1;
        memcpy(buf, out.data(), n);
        buf[n] = 0;
    }
    return out.size() + 1;
}

}  // extern "C"
