// prof.cu -- per-kernel-class launch counters and optional CUDA-event timing
// of every launch on the stream it is launched on (diagnostics for the
// roofline report; no effect on results).
#include <cstdlib>
#include <mutex>
#include <vector>

#include "internal.h"

namespace mpj {

namespace {
struct Pending { int cls; cudaEvent_t a, b; };
std::mutex g_mu;
bool g_on = false;
unsigned long long g_total = 0;
long long g_count[kProfClasses] = {};
double g_ms[kProfClasses] = {};
double g_units[kProfClasses] = {};
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
    if (!g_pool.empty()) { cudaEvent_t e = g_pool.back(); g_pool.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
const char* kNames[kProfClasses] = {
    "solve2_f32", "apply2_f32", "solve2_f64", "apply2_f64", "dgemm_f64", "mgs_panel",
    "mgs_proj", "gram1_f32", "solve1_f32", "apply1_f32", "gram1_f64", "solve1_f64",
    "apply1_f64", "aux", "apply2v_f32", "apply2v_f64", "batched", "tc1_f32", "tc2_f32", "oz_slice", "oz_gemm", "tcv_f32",
    "tcp1_f64", "tcp2_f64", "tcv_f64", "gram_tc64", "tcc_f64", "tcv1_f64", "tile_f32"};
}  // namespace

ProfScope::ProfScope(int cls_, cudaStream_t s_) : cls(cls_), s(s_) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_total += 1;
    g_count[cls] += 1;
    if (g_on) {
        a = take_event();
        if (a) cudaEventRecord(a, s);
    }
}

ProfScope::~ProfScope() {
    if (!a) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t b = take_event();
    if (!b) return;
    cudaEventRecord(b, s);
    g_pending.push_back({cls, a, b});
}

void prof_add_units(int cls, double bytes) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_units[cls] += bytes;
}

// Accumulate the elapsed times of launches whose end events have completed.
void prof_flush() {
    std::lock_guard<std::mutex> lk(g_mu);
    std::vector<Pending> keep;
    for (auto& p : g_pending) {
        if (cudaEventQuery(p.b) != cudaSuccess) { keep.push_back(p); continue; }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) g_ms[p.cls] += ms;
        g_pool.push_back(p.a);
        g_pool.push_back(p.b);
    }
    g_pending.swap(keep);
    cudaGetLastError();   // cudaEventQuery's cudaErrorNotReady is not an error of ours
}

}  // namespace mpj

extern "C" {

void mpj_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(mpj::g_mu);
    mpj::g_on = on != 0;
}

void mpj_profile_reset(void) {
    mpj::prof_flush();
    std::lock_guard<std::mutex> lk(mpj::g_mu);
    for (int i = 0; i < mpj::kProfClasses; ++i) { mpj::g_count[i] = 0; mpj::g_ms[i] = 0.0; mpj::g_units[i] = 0.0; }
}

int mpj_profile_read(int kclass, long long* launches, double* total_ms) {
    if (kclass < 0 || kclass >= mpj::kProfClasses) return MPJ_BAD_ARG;
    mpj::prof_flush();
    std::lock_guard<std::mutex> lk(mpj::g_mu);
    if (launches) *launches = mpj::g_count[kclass];
    if (total_ms) *total_ms = mpj::g_ms[kclass];
    return MPJ_SUCCESS;
}

int mpj_profile_units(int kclass, double* bytes) {
    if (kclass < 0 || kclass >= mpj::kProfClasses || !bytes) return MPJ_BAD_ARG;
    std::lock_guard<std::mutex> lk(mpj::g_mu);
    *bytes = mpj::g_units[kclass];
    return MPJ_SUCCESS;
}

const char* mpj_profile_name(int kclass) {
    if (kclass < 0 || kclass >= mpj::kProfClasses) return "";
    return mpj::kNames[kclass];
}

int mpj_profile_classes(void) { return mpj::kProfClasses; }

unsigned long long mpj_kernel_launches(void) {
    std::lock_guard<std::mutex> lk(mpj::g_mu);
    return mpj::g_total;
}

}  // extern "C"
