// kg_prof.cu -- measurement support: opt-in per-kernel event timing and an
// FP64 throughput probe.  Neither is on the solver path unless switched on.
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "kg_internal.h"

namespace kg {

namespace {
struct Rec {
    int name;
    cudaEvent_t a, b;
};
std::mutex g_pm;
bool g_on = false;
std::vector<std::string> g_names;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
std::vector<std::tuple<std::string, long long, double>> g_result;

cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void recycle() {
    for (auto& r : g_recs) {
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
}
}  // namespace

bool profiling() { return g_on; }

ProfScope::ProfScope(const char* name, cudaStream_t s) : st(s) {
    if (!g_on) return;
    std::lock_guard<std::mutex> lk(g_pm);
    int id = -1;
    for (size_t i = 0; i < g_names.size(); ++i)
        if (g_names[i] == name) id = (int)i;
    if (id < 0) {
        id = (int)g_names.size();
        g_names.push_back(name);
    }
    Rec r{id, take_event(), take_event()};
    cudaEventRecord(r.a, st);
    slot = (int)g_recs.size();
    g_recs.push_back(r);
}

ProfScope::~ProfScope() {
    if (slot < 0) return;
    std::lock_guard<std::mutex> lk(g_pm);
    cudaEventRecord(g_recs[slot].b, st);
}

int profile_start() {
    std::lock_guard<std::mutex> lk(g_pm);
    KG_CUDA(cudaDeviceSynchronize());
    recycle();
    g_names.clear();
    g_result.clear();
    g_on = true;
    return KG_OK;
}

int profile_stop() {
    std::lock_guard<std::mutex> lk(g_pm);
    g_on = false;
    KG_CUDA(cudaDeviceSynchronize());
    std::vector<long long> n(g_names.size(), 0);
    std::vector<double> ms(g_names.size(), 0.0);
    for (auto& r : g_recs) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
            n[r.name] += 1;
            ms[r.name] += t;
        }
    }
    g_result.clear();
    for (size_t i = 0; i < g_names.size(); ++i) g_result.emplace_back(g_names[i], n[i], ms[i]);
    recycle();
    return KG_OK;
}

int profile_count() { return (int)g_result.size(); }

int profile_get(int i, char* name, int len, long long* launches, double* ms) {
    if (i < 0 || i >= (int)g_result.size()) {
        set_error("profile entry %d out of range", i);
        return KG_EINVAL;
    }
    const auto& r = g_result[i];
    if (name && len > 0) {
        std::snprintf(name, len, "%s", std::get<0>(r).c_str());
    }
    if (launches) *launches = std::get<1>(r);
    if (ms) *ms = std::get<2>(r);
    return KG_OK;
}

// Eight independent FMA chains per thread keep the FP64 pipe busy without
// any memory traffic; a never-true test keeps the compiler from dropping them.
__global__ void __launch_bounds__(256) k_fp64_probe(double* out, int iters, double a, double b) {
    double x0 = threadIdx.x * 1e-3, x1 = x0 + 0.1, x2 = x0 + 0.2, x3 = x0 + 0.3;
    double x4 = x0 + 0.4, x5 = x0 + 0.5, x6 = x0 + 0.6, x7 = x0 + 0.7;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b);
        x1 = fma(x1, a, b);
        x2 = fma(x2, a, b);
        x3 = fma(x3, a, b);
        x4 = fma(x4, a, b);
        x5 = fma(x5, a, b);
        x6 = fma(x6, a, b);
        x7 = fma(x7, a, b);
    }
    const double s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == -1.0) out[blockIdx.x] = s;
}

int probe_fp64(double* tflops, cudaStream_t st) {
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    double* out = nullptr;
    KG_CUDA(cudaMalloc(&out, sizeof(double) * nsm * 16));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = nsm * 16, iters = 8192;
    k_fp64_probe<<<blocks, 256, 0, st>>>(out, 256, 0.999999, 1e-7);  // warm-up
    cudaEventRecord(e0, st);
    k_fp64_probe<<<blocks, 256, 0, st>>>(out, iters, 0.999999, 1e-7);
    cudaEventRecord(e1, st);
    const cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return cuda_fail(e, "fp64 probe", __FILE__, __LINE__);
    count_launch(2);
    const double fma_count = (double)blocks * 256.0 * 8.0 * iters;
    *tflops = 2.0 * fma_count / (ms * 1e-3) / 1e12;
    return KG_OK;
}

}  // namespace kg

extern "C" {
int kg_profile_start(void) { return kg::profile_start(); }
int kg_profile_stop(void) { return kg::profile_stop(); }
int kg_profile_count(void) { return kg::profile_count(); }
int kg_profile_get(int i, char* name, int len, long long* launches, double* ms) {
    return kg::profile_get(i, name, len, launches, ms);
}
int kg_probe_fp64(double* tflops, void* stream) {
    if (!tflops) {
        kg::set_error("NULL output");
        return KG_EINVAL;
    }
    return kg::probe_fp64(tflops, (cudaStream_t)stream);
}
}
