// Run-time specialisation of the scan kernel (scan_jit.cuh).
//
// mpm_build compiles the kernel once per distinct filter (q, k, m', symbol
// width, shift, map kind, entry width, table placement) with NVRTC for
// sm_103a, loads the cubin into the device's primary context and keeps it in
// a process-wide cache.  NVRTC is opened with dlopen, so the library loads
// and the generic kernel runs where NVRTC is absent.
#include <dlfcn.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cudaTypedefs.h>
#include <nvrtc.h>

#include "kernels.h"
#include "batch_args.h"
#include "scan_jit_args.h"

namespace mpm {

namespace {

const char kJitSource[] =
#include "scan_jit_src.inc"
    ;
const char kBatchPrelude[] =
#include "batch_prelude_src.inc"
    ;
const char kBatchStage[] =
#include "batch_stage_src.inc"
    ;
const char kBatchKernel[] =
#include "batch_kernel_src.inc"
    ;

struct NvrtcApi {
    bool ok = false;
    nvrtcResult (*create)(nvrtcProgram*, const char*, const char*, int, const char* const*,
                          const char* const*) = nullptr;
    nvrtcResult (*compile)(nvrtcProgram, int, const char* const*) = nullptr;
    nvrtcResult (*log_size)(nvrtcProgram, size_t*) = nullptr;
    nvrtcResult (*log)(nvrtcProgram, char*) = nullptr;
    nvrtcResult (*cubin_size)(nvrtcProgram, size_t*) = nullptr;
    nvrtcResult (*cubin)(nvrtcProgram, char*) = nullptr;
    nvrtcResult (*destroy)(nvrtcProgram*) = nullptr;
};

const NvrtcApi& nvrtc() {
    static NvrtcApi api;
    static std::once_flag once;
    std::call_once(once, [] {
        std::vector<std::string> names;
        if (const char* e = std::getenv("MPM_NVRTC")) names.push_back(e);
        names.push_back("libnvrtc.so.13");
        names.push_back("libnvrtc.so");
        if (const char* e = std::getenv("CUDA_HOME"))
            names.push_back(std::string(e) + "/lib64/libnvrtc.so.13");
        names.push_back("/usr/local/cuda/lib64/libnvrtc.so.13");
        names.push_back("/usr/local/cuda/lib64/libnvrtc.so");
        void* h = nullptr;
        for (auto& n : names)
            if ((h = dlopen(n.c_str(), RTLD_NOW | RTLD_LOCAL))) break;
        if (!h) return;
        api.create = reinterpret_cast<decltype(api.create)>(dlsym(h, "nvrtcCreateProgram"));
        api.compile = reinterpret_cast<decltype(api.compile)>(dlsym(h, "nvrtcCompileProgram"));
        api.log_size = reinterpret_cast<decltype(api.log_size)>(dlsym(h, "nvrtcGetProgramLogSize"));
        api.log = reinterpret_cast<decltype(api.log)>(dlsym(h, "nvrtcGetProgramLog"));
        api.cubin_size = reinterpret_cast<decltype(api.cubin_size)>(dlsym(h, "nvrtcGetCUBINSize"));
        api.cubin = reinterpret_cast<decltype(api.cubin)>(dlsym(h, "nvrtcGetCUBIN"));
        api.destroy = reinterpret_cast<decltype(api.destroy)>(dlsym(h, "nvrtcDestroyProgram"));
        api.ok = api.create && api.compile && api.log_size && api.log && api.cubin_size &&
                 api.cubin && api.destroy;
    });
    return api;
}

struct DriverApi {
    bool ok = false;
    PFN_cuModuleLoadData_v2000 load = nullptr;
    PFN_cuModuleGetFunction_v2000 get = nullptr;
    PFN_cuFuncSetAttribute_v9000 set_attr = nullptr;
    PFN_cuLaunchKernel_v4000 launch = nullptr;
    PFN_cuOccupancyMaxActiveBlocksPerMultiprocessor_v6050 occupancy = nullptr;
    PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
};

template <typename F>
void entry(const char* name, unsigned ver, F* out) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, ver, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        *out = reinterpret_cast<F>(p);
    else
        cudaGetLastError();
}

const DriverApi& driver() {
    static DriverApi api;
    static std::once_flag once;
    std::call_once(once, [] {
        entry("cuModuleLoadData", 2000, &api.load);
        entry("cuModuleGetFunction", 2000, &api.get);
        entry("cuFuncSetAttribute", 9000, &api.set_attr);
        entry("cuLaunchKernel", 4000, &api.launch);
        entry("cuOccupancyMaxActiveBlocksPerMultiprocessor", 6050, &api.occupancy);
        entry("cuTensorMapEncodeTiled", 12000, &api.encode);
        api.ok = api.load && api.get && api.set_attr && api.launch && api.occupancy && api.encode;
    });
    return api;
}

uint32_t gcd_u(uint32_t a, uint32_t b) {
    while (b) {
        uint32_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

uint32_t lcm_u(uint32_t a, uint32_t b) { return a / gcd_u(a, b) * b; }

constexpr size_t kSmemLimit = 227 * 1024;

}  // namespace

// Compile-time constants of one specialisation and its launch geometry.
struct JitSpec {
    int q, k, mp, ell, shift, mode, eb, smem, table_bytes, C, S, warps, verify, ecap, ov, ebits;
    size_t smem_bytes;

    std::string defines() const {
        char buf[640];
        std::snprintf(buf, sizeof(buf),
                      "-DMPM_Q=%d -DMPM_K=%d -DMPM_MP=%d -DMPM_ELL=%d -DMPM_SHIFT=%d "
                      "-DMPM_MODE=%d -DMPM_EB=%d -DMPM_SMEM=%d -DMPM_TABLE_BYTES=%du "
                      "-DMPM_C=%d -DMPM_S=%d -DMPM_WARPS=%d -DMPM_VERIFY=%d -DMPM_EMIT_CAP=%d "
                      "-DMPM_OV=%d -DMPM_EBITS=%d",
                      q, k, mp, ell, shift, mode, eb, smem, table_bytes, C, S, warps, verify,
                      ecap, ov, ebits);
        return buf;
    }
};

struct JitKernel {
    JitSpec spec;
    CUfunction fn = nullptr;
    int blocks_per_sm = 1;
};

// Stage bytes of the specialised scans for P text bytes per sampled q-gram:
// rows of at least 80 bytes (48-byte rows measured up to 3x slower on
// GB300); odd multiples of lcm(P, 16) keep C/16 odd, which keeps the 16-byte
// shared loads of a quarter warp on distinct banks; non-overlapping, at
// most 64 report bits per stage (C / P * k <= 64; the overlapping stage finds
// its report bits again only when one fired).  0 when lcm(P, 16) > 256.
uint32_t jit_stage_bytes(uint32_t P, int k, bool overlap) {
    const uint32_t base = lcm_u(P, 16);
    if (base > 256) return 0;
    auto bits_ok = [&](uint32_t c) { return overlap || c / P * (uint32_t)k <= 64; };
    uint32_t C = base;
    const uint32_t step = ((base / 16) % 2 == 1) ? 2 * base : base;
    while (C < 80 && C + step <= 256 && bits_ok(C + step)) C += step;
    return bits_ok(C) ? C : 0;
}

// The specialisation for a filter, or false when the filter is outside what
// the specialised kernel handles (then the generic kernel runs).
bool jit_spec(const FilterDev& f, bool verify, JitSpec* out) {
    JitSpec s{};
    s.verify = verify ? 1 : 0;
    s.ecap = 64;
    s.q = f.q;
    s.k = f.k;
    s.mp = f.mprime;
    s.ell = f.ell;
    s.shift = f.map_kind == MPM_MAP_LOWBITS ? f.shift : 0;
    s.mode = f.map_kind == MPM_MAP_LOWBITS ? 0 : (f.map_kind == MPM_MAP_QHASH ? 2 : 1);
    s.eb = f.entry_bytes;
    s.ebits = f.entry_bits > 0 ? f.entry_bits : 8 * f.entry_bytes;
    s.smem = f.smem_table ? 1 : 0;
    s.table_bytes = f.smem_table ? (int)f.table_bytes : 0;
    s.ov = f.overlap ? 1 : 0;
    // bytes per sampled q-gram: k q non-overlapping, k overlapping
    const uint32_t P = (uint32_t)(s.ov ? f.k : f.k * f.q);
    const uint32_t base = lcm_u(P, 16);
    uint32_t C = jit_stage_bytes(P, f.k, s.ov != 0);
    if (C == 0) return false;
    auto bits_ok = [&](uint32_t c) { return s.ov || c / P * (uint32_t)f.k <= 64; };
    s.warps = 16;
    // overrides for tuning the geometry: MPM_JIT_C (stage bytes, a multiple
    // of lcm(k q, 16) up to 256) and MPM_JIT_WARPS (4..32)
    if (const char* e = std::getenv("MPM_JIT_C")) {
        const uint32_t c = (uint32_t)std::atoi(e);
        if (c >= base && c <= 256 && c % base == 0) C = c;
    }
    if (const char* e = std::getenv("MPM_JIT_WARPS")) {
        const int w = std::atoi(e);
        if (w >= 4 && w <= 32) s.warps = w;
    }
    if (!bits_ok(C)) return false;
    s.C = (int)C;
    for (;;) {
        const size_t fixed =
            (size_t)s.table_bytes + 256 + 8 * s.warps * 4 + 8 * s.warps * s.ecap + 128;
        const size_t per_stage = (size_t)s.warps * 32 * C;
        const size_t budget = kSmemLimit > fixed ? kSmemLimit - fixed : 0;
        s.S = (int)std::min<size_t>(4, budget / per_stage);
        if (s.S >= 2) break;
        if (s.warps <= 4) return false;
        s.warps /= 2;
    }
    const size_t emit_off = (size_t)s.table_bytes + 256 + 8 * s.warps * s.S;
    const size_t stage_off = (emit_off + 8 * s.warps * s.ecap + 127) / 128 * 128;
    s.smem_bytes = stage_off + (size_t)s.warps * s.S * 32 * C;
    *out = s;
    return true;
}

// Compiles a source text with NVRTC for sm_103a, with the -D options in
// `defines` (space separated); the cubin (may be null) and the log.
static int compile_source(const char* src, const char* name, const std::string& defines,
                          std::string* cubin, std::string* log) {
    const NvrtcApi& nv = nvrtc();
    if (!nv.ok) {
        if (log) *log = "NVRTC not found";
        return MPM_ENOTSUP;
    }
    nvrtcProgram prog;
    if (nv.create(&prog, src, name, 0, nullptr, nullptr) != NVRTC_SUCCESS) return MPM_ECUDA;
    std::vector<std::string> opts = {"--gpu-architecture=sm_103a", "--std=c++17", "-lineinfo"};
    if (std::getenv("MPM_JIT_VERBOSE")) opts.push_back("--ptxas-options=-v");
    {
        const std::string& d = defines;
        size_t pos = 0;
        while (pos < d.size()) {
            size_t e = d.find(' ', pos);
            if (e == std::string::npos) e = d.size();
            if (e > pos) opts.push_back(d.substr(pos, e - pos));
            pos = e + 1;
        }
    }
    std::vector<const char*> argv;
    for (auto& o : opts) argv.push_back(o.c_str());
    const nvrtcResult rc = nv.compile(prog, (int)argv.size(), argv.data());
    size_t ls = 0;
    nv.log_size(prog, &ls);
    if (log) {
        log->assign(ls, '\0');
        if (ls) nv.log(prog, &(*log)[0]);
    }
    int ret = MPM_OK;
    if (rc != NVRTC_SUCCESS) {
        ret = MPM_ECUDA;
    } else if (cubin) {
        size_t cs = 0;
        nv.cubin_size(prog, &cs);
        cubin->assign(cs, '\0');
        if (!cs || nv.cubin(prog, &(*cubin)[0]) != NVRTC_SUCCESS) ret = MPM_ECUDA;
    }
    nv.destroy(&prog);
    return ret;
}

static int compile_spec(const JitSpec& s, std::string* cubin, std::string* log) {
    return compile_source(kJitSource, "mpm_scan_jit.cu", s.defines(), cubin, log);
}

int jit_compile_only(const FilterDev& f, bool verify, std::string* log) {
    JitSpec s;
    if (!jit_spec(f, verify, &s)) {
        if (log) *log = "filter outside the specialised kernel";
        return MPM_ENOTSUP;
    }
    std::string cubin;
    return compile_spec(s, &cubin, log);
}

namespace {
std::mutex g_cache_mu;
std::map<std::string, std::unique_ptr<JitKernel>> g_cache;  // loaded kernels
std::map<std::string, std::string> g_cubins;               // compiled, not yet loaded
}  // namespace

void jit_precompile(const std::vector<FilterDev>& fs, bool verify, int threads) {
    std::vector<JitSpec> todo;
    {
        std::lock_guard<std::mutex> lock(g_cache_mu);
        std::map<std::string, bool> seen;
        for (const auto& f : fs) {
            JitSpec s;
            if (!jit_spec(f, verify, &s)) continue;
            const std::string d = s.defines();
            if (g_cubins.count(d) || seen.count(d)) continue;
            seen[d] = true;
            todo.push_back(s);
        }
    }
    if (todo.empty() || !nvrtc().ok) return;
    std::vector<std::string> out(todo.size());
    std::vector<int> rc(todo.size(), MPM_ECUDA);
    size_t next = 0;
    std::mutex next_mu;
    auto work = [&] {
        for (;;) {
            size_t i;
            {
                std::lock_guard<std::mutex> lock(next_mu);
                if (next >= todo.size()) return;
                i = next++;
            }
            rc[i] = compile_spec(todo[i], &out[i], nullptr);
        }
    };
    std::vector<std::thread> pool;
    for (int t = 0; t < std::max(1, threads); t++) pool.emplace_back(work);
    for (auto& t : pool) t.join();
    std::lock_guard<std::mutex> lock(g_cache_mu);
    for (size_t i = 0; i < todo.size(); i++)
        if (rc[i] == MPM_OK) g_cubins[todo[i].defines()] = std::move(out[i]);
}

const JitKernel* jit_scan_kernel(const FilterDev& f, bool verify, int device, int* err,
                                 std::string* log) {
    auto& mu = g_cache_mu;
    auto& cache = g_cache;
    *err = MPM_OK;
    JitSpec s;
    if (!jit_spec(f, verify, &s)) {
        *err = MPM_ENOTSUP;
        return nullptr;
    }
    const DriverApi& drv = driver();
    if (!drv.ok) {
        *err = MPM_ENOTSUP;
        return nullptr;
    }
    const std::string key = std::to_string(device) + " " + s.defines();
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second.get();
    std::string cubin;
    auto pre = g_cubins.find(s.defines());
    if (pre != g_cubins.end()) {
        cubin = pre->second;
    } else {
        int rc = compile_spec(s, &cubin, log);
        if (rc) {
            *err = rc;
            return nullptr;
        }
        g_cubins[s.defines()] = cubin;
    }
    CUmodule mod;
    CUfunction fn;
    // the module goes into the device's primary context, which the runtime
    // creates on its first call that needs one
    cudaFree(nullptr);
    if (drv.load(&mod, cubin.data()) != CUDA_SUCCESS ||
        drv.get(&fn, mod, "mpm_scan_jit") != CUDA_SUCCESS ||
        drv.set_attr(fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, (int)s.smem_bytes) !=
            CUDA_SUCCESS) {
        *err = MPM_ECUDA;
        return nullptr;
    }
    auto k = std::make_unique<JitKernel>();
    k->spec = s;
    k->fn = fn;
    int per_sm = 0;
    if (drv.occupancy(&per_sm, fn, s.warps * 32, s.smem_bytes) != CUDA_SUCCESS || per_sm < 1)
        per_sm = 1;
    k->blocks_per_sm = per_sm;
    const JitKernel* out = k.get();
    cache.emplace(key, std::move(k));
    return out;
}

bool jit_verifies(const JitKernel* k) { return k && k->spec.verify; }

namespace {
std::atomic<int> g_injected_fault{0};
}  // namespace

// Test hook (mpm_test_inject): a fault armed for the next specialised scan.
int take_injected_fault() { return g_injected_fault.exchange(0); }
void set_injected_fault(int f) { g_injected_fault.store(f); }

int launch_scan_jit(const ScanArgs& A, const VerifyArgs* V, const JitKernel* K, int num_sms,
                    int chunk, cudaStream_t stream) {
    if (A.n == 0) return 0;
    const DriverApi& drv = driver();
    const JitSpec& s = K->spec;
    const uint32_t n = A.n;
    const uint32_t C = (uint32_t)s.C;
    const uint32_t P = (uint32_t)(s.ov ? s.k : s.k * s.q);
    // one block per SM but one: the SM left over takes the closing kernels
    // of pipelined searches (side stream) without delaying a persistent scan
    // block, whose rows no other block takes over (measured: 1.5 % faster
    // pipelined steps than a block on every SM)
    uint32_t blocks = (uint32_t)((num_sms > 8 ? num_sms - 1 : num_sms) * K->blocks_per_sm);
    // measurement override: the number of blocks (MPM_JIT_GRID)
    if (const char* e = std::getenv("MPM_JIT_GRID")) {
        const int g = std::atoi(e);
        if (g >= 1 && g <= 4 * num_sms * K->blocks_per_sm) blocks = (uint32_t)g;
    }
    const uint32_t GW = blocks * (uint32_t)s.warps;
    // bytes of the samples before a row (overlapping: and a sample's first
    // q-1 bytes), in whole stages
    const uint32_t wb = (uint32_t)((s.mp - 1) * (int)P + (s.ov ? s.q - 1 : 0));
    const uint32_t warm = (wb + C - 1) / C * C;
    const uint32_t row_warps = GW > 1 ? GW - 1 : 1;
    uint64_t Lst = chunk > 0 ? (uint64_t)chunk : ((uint64_t)n + 32ull * row_warps - 1) / (32ull * row_warps);
    Lst = (Lst + C - 1) / C * C;
    Lst = std::max<uint64_t>(Lst, std::max<uint64_t>(4ull * C, warm + C));
    const bool aligned = (reinterpret_cast<uintptr_t>(A.T) & 15) == 0;
    const uint64_t R = aligned ? n / Lst : 0;

    JitScanArgs J{};
    J.inject = (uint32_t)take_injected_fault();
    J.T = A.T;
    J.table = A.f.table;
    J.mu = A.f.mu;
    J.cand = reinterpret_cast<unsigned long long*>(A.cand);
    J.counters = A.counters;
    J.n = n;
    J.cap = A.cap;
    J.Lst = (uint32_t)Lst;
    J.R = (uint32_t)R;
    J.RG = (uint32_t)((R + 31) / 32);
    J.row_warps = row_warps;
    J.pa = (uint32_t)(R * Lst);
    const uint32_t rest = n - J.pa;
    const uint32_t lanes = R > 0 ? 32u : GW * 32u;
    uint32_t Ls = (rest + lanes - 1) / lanes;
    Ls = std::max<uint32_t>((Ls + P - 1) / P * P, 4 * P);
    J.Ls = Ls;
    J.nstreams = rest ? (rest + Ls - 1) / Ls : 0;
    if (s.verify) {
        if (!V) return -1;
        J.m = V->m;
        J.slots = V->slots;
        J.pat = V->pat;
        J.pid = V->pid;
        J.pat_off = V->pat_off;
        J.occ = reinterpret_cast<unsigned long long*>(V->occ);
        J.slot_mask = V->slot_mask;
        J.key_bytes = (uint32_t)V->key_bytes;
        J.occ_cap = V->occ_cap;
    }

    alignas(64) CUtensorMap tmap;
    std::memset(&tmap, 0, sizeof(tmap));
    if (R > 0) {
        cuuint64_t dims[2] = {Lst, R};
        cuuint64_t strides[1] = {Lst};
        cuuint32_t box[2] = {C, 32};
        cuuint32_t estr[2] = {1, 1};
        if (drv.encode(&tmap, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(A.T), dims,
                       strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return -1;
    }
    void* params[2] = {&J, &tmap};
    if (drv.launch(K->fn, blocks, 1, 1, (unsigned)(s.warps * 32), 1, 1, (unsigned)s.smem_bytes,
                   reinterpret_cast<CUstream>(stream), params, nullptr) != CUDA_SUCCESS)
        return -1;
    return 1;
}

// ------------------------------------------------------- the batched kernel

// Dynamic shared memory of the batched kernel: the byte map, the largest mask
// table it copies, the largest key bitmap.
constexpr size_t kBatchJitSmem = 256 + kBatchSmemTable + kBatchKeyBits / 8;

struct BatchJit {
    CUfunction fn = nullptr;
    int warps = 16;  // per block, as compiled
};

// Warps per block of the batched kernel: 24 (measured on the batch-4096
// workload: 16 warps 1.92 ms, 24 warps 1.82 ms, 32 warps 1.89 ms per scan;
// measurement override MPM_BATCH_WARPS: 8, 16, 24 or 32).
static int batch_warps() {
    if (const char* e = std::getenv("MPM_BATCH_WARPS")) {
        const int w = std::atoi(e);
        if (w == 8 || w == 16 || w == 24 || w == 32) return w;
    }
    return 24;
}

namespace {
std::mutex g_batch_mu;
std::map<std::string, std::string> g_batch_cubins;                // source -> cubin
std::map<std::string, std::unique_ptr<BatchJit>> g_batch_kernels;  // device + source -> kernel
}  // namespace

// The batch's source: the prelude, then for every parameter set its stage
// primitives and lane scan in a namespace bv<i> of their own, compiled with
// its constants, then the kernel dispatching on the set's variant index.
static std::string batch_source(const std::vector<BatchVariant>& vs) {
    char buf[512];
    // stages a lane prefetches into L2 ahead of its loads (6; measurement
    // override MPM_BATCH_PREFETCH, 0..8)
    int prefetch = 6;
    if (const char* e = std::getenv("MPM_BATCH_PREFETCH")) {
        const int v = std::atoi(e);
        if (v >= 0 && v <= 8) prefetch = v;
    }
    std::snprintf(buf, sizeof(buf), "#define MPM_BATCH_PREFETCH %d\n#define MPM_BATCH_WARPS %d\n",
                  prefetch, batch_warps());
    std::string src = buf;
    src += kBatchPrelude;
    for (size_t i = 0; i < vs.size(); i++) {
        const BatchVariant& v = vs[i];
        std::snprintf(buf, sizeof(buf),
                      "namespace mpm {\nnamespace bv%zu {\n#define MPM_Q %d\n#define MPM_K %d\n"
                      "#define MPM_MP %d\n#define MPM_ELL %d\n#define MPM_SHIFT %d\n"
                      "#define MPM_MODE %d\n#define MPM_EB %d\n#define MPM_SMEM %d\n"
                      "#define MPM_C %u\n#define MPM_OV 0\n#define MPM_STAGES %d\n"
                      "#define MPM_EBITS %d\n",
                      i, v.q, v.k, v.mp, v.ell, v.shift, v.mode, v.eb, v.smem, v.C, v.stages,
                      v.ebits);
        src += buf;
        src += kBatchStage;
        src += "\n#undef MPM_Q\n#undef MPM_K\n#undef MPM_MP\n#undef MPM_ELL\n#undef MPM_SHIFT\n"
               "#undef MPM_MODE\n#undef MPM_EB\n#undef MPM_SMEM\n#undef MPM_C\n#undef MPM_OV\n"
               "#undef MPM_STAGES\n#undef MPM_EBITS\n"
               "}  // namespace bv\n}  // namespace mpm\n";
    }
    src += "#define MPM_BATCH_CASES";
    for (size_t i = 0; i < vs.size(); i++) {
        std::snprintf(buf, sizeof(buf), " CASE(%zu)", i);
        src += buf;
    }
    src += "\n";
    src += kBatchKernel;
    return src;
}

static int batch_cubin(const std::string& src, std::string* cubin, std::string* log) {
    {
        std::lock_guard<std::mutex> lock(g_batch_mu);
        auto it = g_batch_cubins.find(src);
        if (it != g_batch_cubins.end()) {
            *cubin = it->second;
            return MPM_OK;
        }
    }
    const int rc = compile_source(src.c_str(), "mpm_batch_jit.cu", "", cubin, log);
    if (rc == MPM_OK) {
        std::lock_guard<std::mutex> lock(g_batch_mu);
        g_batch_cubins[src] = *cubin;
    }
    return rc;
}

void jit_batch_precompile(const std::vector<BatchVariant>& vs, int threads) {
    if (!nvrtc().ok) return;
    std::vector<std::string> todo;
    {
        std::lock_guard<std::mutex> lock(g_batch_mu);
        for (const auto& v : vs) {
            std::string src = batch_source(std::vector<BatchVariant>{v});
            if (!g_batch_cubins.count(src) && std::find(todo.begin(), todo.end(), src) == todo.end())
                todo.push_back(std::move(src));
        }
    }
    size_t next = 0;
    std::mutex next_mu;
    auto work = [&] {
        for (;;) {
            size_t i;
            {
                std::lock_guard<std::mutex> lock(next_mu);
                if (next >= todo.size()) return;
                i = next++;
            }
            std::string cubin;
            batch_cubin(todo[i], &cubin, nullptr);
        }
    };
    std::vector<std::thread> pool;
    for (int t = 0; t < std::max(1, threads); t++) pool.emplace_back(work);
    for (auto& t : pool) t.join();
}

int jit_batch_compile_only(const std::vector<BatchVariant>& vs, std::string* log) {
    std::string cubin;
    return batch_cubin(batch_source(vs), &cubin, log);
}

const BatchJit* jit_batch_kernel(const std::vector<BatchVariant>& vs, int device, int* err,
                                 std::string* log) {
    *err = MPM_OK;
    const DriverApi& drv = driver();
    if (!drv.ok || vs.empty()) {
        *err = MPM_ENOTSUP;
        return nullptr;
    }
    const std::string src = batch_source(vs);
    const std::string key = std::to_string(device) + "\n" + src;
    {
        std::lock_guard<std::mutex> lock(g_batch_mu);
        auto it = g_batch_kernels.find(key);
        if (it != g_batch_kernels.end()) return it->second.get();
    }
    std::string cubin;
    const int rc = batch_cubin(src, &cubin, log);
    if (rc) {
        *err = rc;
        return nullptr;
    }
    CUmodule mod;
    CUfunction fn;
    cudaFree(nullptr);  // the primary context, as for the single-text scan
    if (drv.load(&mod, cubin.data()) != CUDA_SUCCESS ||
        drv.get(&fn, mod, "mpm_batch_jit") != CUDA_SUCCESS ||
        drv.set_attr(fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, (int)kBatchJitSmem) !=
            CUDA_SUCCESS) {
        *err = MPM_ECUDA;
        return nullptr;
    }
    auto k = std::make_unique<BatchJit>();
    k->fn = fn;
    k->warps = batch_warps();
    std::lock_guard<std::mutex> lock(g_batch_mu);
    auto& slot = g_batch_kernels[key];
    if (!slot) slot = std::move(k);
    return slot.get();
}

int launch_batch_jit(const BatchJit* k, const BatchJitArgs& a, int num_sms, cudaStream_t s) {
    const DriverApi& drv = driver();
    BatchJitArgs args = a;
    void* params[1] = {&args};
    // one block per SM (the kernel's launch bounds)
    if (drv.launch(k->fn, (unsigned)num_sms, 1, 1, (unsigned)(32 * k->warps), 1, 1,
                   (unsigned)kBatchJitSmem,
                   reinterpret_cast<CUstream>(s), params, nullptr) != CUDA_SUCCESS)
        return -1;
    return 1;
}

}  // namespace mpm

extern "C" int mpm_test_inject(int fault) {
    if (fault < 0 || fault > 1) return mpm::set_error(MPM_EINVAL);
    mpm::set_injected_fault(fault);
    return mpm::set_error(MPM_OK);
}
