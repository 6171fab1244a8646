#include <cuda_runtime.h>
thread_local emu_uint3 threadIdx, blockIdx;
thread_local dim3 blockDim, gridDim;
thread_local unsigned char *emu_dyn_smem_ptr;
static int g_nsm = 4;
int emu_nsm() { const char *s = getenv("EMU_NSM"); return s ? atoi(s) : g_nsm; }
std::mutex &emu_atomic_mutex() { static std::mutex m; return m; }

struct Barrier {
    std::mutex m; std::condition_variable cv; int n = 0, count = 0; uint64_t gen = 0;
    void init(int k) { n = k; count = 0; }
    void wait() {
        std::unique_lock<std::mutex> l(m);
        uint64_t g = gen;
        if (++count == n) { count = 0; ++gen; cv.notify_all(); return; }
        if (!cv.wait_for(l, std::chrono::seconds(20), [&] { return gen != g; })) {
            fprintf(stderr, "EMU DEADLOCK: barrier of %d waited 20 s (t=%u b=%u)\n", n, threadIdx.x, blockIdx.x);
            abort();
        }
    }
};
struct WarpState {
    std::mutex m;
    std::map<unsigned, std::unique_ptr<Barrier>> bars;
    uint64_t buf[32];
    Barrier &bar(unsigned mask) {
        std::lock_guard<std::mutex> g(m);
        auto &p = bars[mask];
        if (!p) { p = std::make_unique<Barrier>(); p->init(__builtin_popcount(mask)); }
        return *p;
    }
};
static Barrier g_block_bar;
static std::vector<std::unique_ptr<WarpState>> g_warps;
static int g_block_threads;

void emu_syncthreads() { g_block_bar.wait(); }
static WarpState &my_warp() { return *g_warps[threadIdx.x / 32]; }
static void check_mask(unsigned mask) {
    const int l = threadIdx.x & 31;
    const int nw_lanes = std::min(32, g_block_threads - (int)(threadIdx.x / 32) * 32);
    const unsigned valid = nw_lanes >= 32 ? 0xffffffffu : ((1u << nw_lanes) - 1u);
    if (!((mask >> l) & 1u)) { fprintf(stderr, "EMU: lane %d not in mask %08x\n", l, mask); abort(); }
    if (mask & ~valid) { fprintf(stderr, "EMU: mask %08x names lanes beyond the block\n", mask); abort(); }
}
void emu_warp_sync(unsigned mask) { check_mask(mask); my_warp().bar(mask).wait(); }
uint64_t emu_warp_xchg(unsigned mask, uint64_t v, int src) {
    check_mask(mask);
    WarpState &w = my_warp();
    Barrier &b = w.bar(mask);
    w.buf[threadIdx.x & 31] = v;
    b.wait();
    if (!((mask >> src) & 1u)) { fprintf(stderr, "EMU: shuffle source lane %d outside mask %08x\n", src, mask); abort(); }
    uint64_t r = w.buf[src];
    b.wait();
    return r;
}
unsigned emu_match_any(unsigned mask, uint64_t key) {
    check_mask(mask);
    WarpState &w = my_warp();
    Barrier &b = w.bar(mask);
    w.buf[threadIdx.x & 31] = key;
    b.wait();
    unsigned r = 0;
    for (int l = 0; l < 32; ++l)
        if (((mask >> l) & 1u) && w.buf[l] == key) r |= 1u << l;
    b.wait();
    return r;
}
void emu_run_grid(const EmuCfg &c, const std::function<void()> &f) {
    const int nt = (int)(c.b.x * c.b.y * c.b.z);
    if (nt <= 0 || nt > 1024) { fprintf(stderr, "EMU: bad block size %d\n", nt); abort(); }
    if (c.smem > 232448) { fprintf(stderr, "EMU: dynamic smem %zu too large\n", c.smem); abort(); }
    for (unsigned bz = 0; bz < c.g.z; ++bz)
        for (unsigned by = 0; by < c.g.y; ++by)
            for (unsigned bx = 0; bx < c.g.x; ++bx) {
                std::vector<unsigned char> dyn(c.smem ? c.smem : 1);
                unsigned char *dp = (unsigned char *)malloc(c.smem ? c.smem : 1);
                memset(dp, 0x5A, c.smem ? c.smem : 1);
                g_block_bar.init(nt);
                g_block_threads = nt;
                g_warps.clear();
                for (int w = 0; w < (nt + 31) / 32; ++w) g_warps.push_back(std::make_unique<WarpState>());
                std::vector<std::thread> th;
                th.reserve(nt);
                for (int t = 0; t < nt; ++t)
                    th.emplace_back([&, t] {
                        threadIdx.x = t % c.b.x; threadIdx.y = (t / c.b.x) % c.b.y; threadIdx.z = t / (c.b.x * c.b.y);
                        blockIdx.x = bx; blockIdx.y = by; blockIdx.z = bz;
                        blockDim = c.b; gridDim = c.g;
                        emu_dyn_smem_ptr = dp;
                        f();
                    });
                for (auto &x : th) x.join();
                free(dp);
            }
}
