// Run-time specialisation of the fused detection kernel.
//
// The kernel source (detect_kernel.cuh, embedded at build time) is compiled
// by NVRTC for sm_103a once per (ladder radii, tile configuration, mode,
// store flag), with the radii baked in as compile-time constants so that the
// scale and tap loops unroll completely.  Cubins are cached on disk (keyed by
// a hash of the full source text and options) and modules per device in
// process memory.
#include <dlfcn.h>
#include <nvrtc.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>

#include "internal.h"

namespace mhfd {

namespace {

#include "kernel_src.inc"  // kTypesSrc, kKernelSrc

constexpr int kSmemLimit = kSmemLimitBytes;

std::mutex g_mu;
std::map<std::string, Variant *> g_variants;

unsigned long long fnv1a(const std::string &s) {
    unsigned long long h = 1469598103934665603ull;
    for (unsigned char c : s) {
        h ^= c;
        h *= 1099511628211ull;
    }
    return h;
}

std::string lib_dir() {
    Dl_info info;
    if (dladdr(reinterpret_cast<void *>(&fnv1a), &info) && info.dli_fname) {
        std::string p(info.dli_fname);
        const size_t k = p.rfind('/');
        if (k != std::string::npos) return p.substr(0, k);
    }
    return ".";
}

std::string cache_dir() {
    const char *e = std::getenv("MHFD_JIT_CACHE");
    std::string d = (e && *e) ? std::string(e) : lib_dir() + "/_jit_cache";
    mkdir(d.c_str(), 0755);
    return d;
}

std::string join(const std::vector<int> &v) {
    std::ostringstream o;
    for (size_t i = 0; i < v.size(); ++i) o << (i ? "," : "") << v[i];
    return o.str();
}

std::string join_f(const std::vector<float> &v) {
    std::string o;
    char buf[64];
    for (size_t i = 0; i < v.size(); ++i) {
        std::snprintf(buf, sizeof(buf), "%s%af", i ? "," : "", (double)v[i]);
        o += buf;
    }
    return o;
}

std::string make_source(const LadderKey &lk, int mode, int store, const TileConfig &c) {
    const std::vector<int> &R = lk.R;
    const int smode = mode | (lk.response ? kModeLog : 0);
    std::ostringstream o;
    o << "#define MHFD_NL " << R.size() << "\n"
      << "#define MHFD_RLIST " << join(R) << "\n"
      << "#define MHFD_TAPS " << join_f(lk.taps) << "\n"
      << "#define MHFD_TSC " << join_f(lk.tsc) << "\n"
      << "#define MHFD_NGROUPS " << (c.gb.size() - 1) << "\n"
      << "#define MHFD_GB " << join(c.gb) << "\n"
      << "#define MHFD_TX2 " << c.tx2 << "\n"
      << "#define MHFD_TY2 " << c.ty2 << "\n"
      << "#define MHFD_BROWS " << brows_for(R, smode, c) << "\n"
      << "#define MHFD_RB " << c.rb << "\n"
      << "#define MHFD_HR " << ((mode & 3) <= 1 ? item_rows(c) : 1) << "\n"
      << "#define MHFD_HW " << ((mode & 3) <= 1 ? item_cols(c) : 4) << "\n"
      << "#define MHFD_VTC " << c.tc << "\n"
      << "#define MHFD_NT " << c.nt << "\n"
      << "#define MHFD_MODE " << mode << "\n"
      << "#define MHFD_STORE " << store << "\n"
      << "#define MHFD_BOUNDARY " << lk.boundary << "\n"
      << "#define MHFD_RESPONSE " << lk.response << "\n"
      << "#define MHFD_TAPS2 " << (lk.response ? join_f(lk.taps2) : std::string("0.0f")) << "\n";
    // MHFD_DEBUG_CHECKS=1: the debug build of the kernel, whose indices are
    // checked against their buffers (a failure is reported as MHFD_ERR_CHECK)
    if (const char *e = std::getenv("MHFD_DEBUG_CHECKS"))
        if (e[0] == '1') o << "#define MHFD_CHECKS 1\n";
    // the kernel's own shared-memory layout must be the one the host sized
    // and chose the tile by: a compile error otherwise
    const std::string check = "\nstatic_assert(mk::SMEM_BYTES == " +
                              std::to_string(smem_estimate(R, smode, c)) +
                              ", \"kernel shared-memory layout differs from the host estimate\");\n";
    return o.str() + kTypesSrc + kKernelSrc + check;
}

const char *kOpts[] = {"--gpu-architecture=sm_103a", "--std=c++17", "-lineinfo"};

bool read_file(const std::string &path, std::string *out) {
    std::ifstream f(path, std::ios::binary);
    if (!f) return false;
    std::ostringstream ss;
    ss << f.rdbuf();
    *out = ss.str();
    return !out->empty();
}

void write_file_atomic(const std::string &path, const std::string &data) {
    const std::string tmp = path + ".tmp." + std::to_string(getpid());
    {
        std::ofstream f(tmp, std::ios::binary);
        if (!f) return;
        f.write(data.data(), (std::streamsize)data.size());
    }
    std::rename(tmp.c_str(), path.c_str());
}

int compile_cubin(const std::string &src, std::string *cubin) {
    // MHFD_JIT_DUMP=<dir>: also write each compiled source there (to inspect
    // register use with nvcc -Xptxas -v)
    if (const char *dump = std::getenv("MHFD_JIT_DUMP")) {
        if (*dump) {
            char name[64];
            std::snprintf(name, sizeof(name), "/mhfd_%016llx.cu", fnv1a(src));
            write_file_atomic(std::string(dump) + name, src);
        }
    }
    nvrtcProgram prog;
    nvrtcResult r = nvrtcCreateProgram(&prog, src.c_str(), "mhfd_fused.cu", 0, nullptr, nullptr);
    if (r != NVRTC_SUCCESS) return fail(MHFD_ERR_JIT, std::string("nvrtcCreateProgram: ") + nvrtcGetErrorString(r));
    r = nvrtcCompileProgram(prog, (int)(sizeof(kOpts) / sizeof(kOpts[0])), kOpts);
    if (r != NVRTC_SUCCESS) {
        size_t n = 0;
        nvrtcGetProgramLogSize(prog, &n);
        std::string log(n, '\0');
        if (n) nvrtcGetProgramLog(prog, &log[0]);
        nvrtcDestroyProgram(&prog);
        if (log.size() > 4000) log = log.substr(0, 4000);
        return fail(MHFD_ERR_JIT, "NVRTC compile failed: " + log);
    }
    size_t n = 0;
    nvrtcGetCUBINSize(prog, &n);
    cubin->assign(n, '\0');
    nvrtcGetCUBIN(prog, &(*cubin)[0]);
    nvrtcDestroyProgram(&prog);
    return MHFD_OK;
}

int drv_fail(CUresult r, const char *what) {
    const char *s = nullptr;
    if (drv().getErrorString) drv().getErrorString(r, &s);
    return fail(MHFD_ERR_CUDA, std::string(what) + ": " + (s ? s : "unknown driver error"));
}

template <class F>
void resolve(const char *name, F *fp, bool *ok) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, 13000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p) {
        *ok = false;
        *fp = nullptr;
        return;
    }
    *fp = reinterpret_cast<F>(p);
}

}  // namespace

const DrvApi &drv() {
    static DrvApi api = [] {
        DrvApi a;
        std::memset(&a, 0, sizeof(a));
        a.ok = true;
        resolve("cuModuleLoadData", &a.moduleLoadData, &a.ok);
        resolve("cuModuleUnload", &a.moduleUnload, &a.ok);
        resolve("cuModuleGetFunction", &a.moduleGetFunction, &a.ok);
        resolve("cuModuleGetGlobal", &a.moduleGetGlobal, &a.ok);
        resolve("cuMemcpyDtoH", &a.memcpyDtoH, &a.ok);
        resolve("cuFuncSetAttribute", &a.funcSetAttribute, &a.ok);
        resolve("cuLaunchKernel", &a.launchKernel, &a.ok);
        resolve("cuGetErrorString", &a.getErrorString, &a.ok);
        resolve("cuOccupancyMaxActiveBlocksPerMultiprocessor", &a.occupancy, &a.ok);
        return a;
    }();
    return api;
}

namespace {

// `mode` is the kernel mode (0 paper rule, 1 26-neighbour rule, 2 soft
// forward, 3 level blur) plus kModeLog for the LoG response, whose levels
// need one more halo pixel and two V rows each, and whose layers are the
// levels themselves (not their differences).
bool is_log(int mode) { return (mode & kModeLog) != 0; }

int rmax_of(const std::vector<int> &R) {
    int m = 0;
    for (int r : R) m = r > m ? r : m;
    return m;
}

int halo_of(const std::vector<int> &R, int mode) { return rmax_of(R) + (is_log(mode) ? 1 : 0); }

// bytes of everything but the input window
int smem_fixed(const std::vector<int> &R, int mode, const TileConfig &c) {
    const bool log = is_log(mode);
    const int base = mode & 3;
    const int layers = log ? (int)R.size() : (int)R.size() - 1;
    int vrow = 0;
    for (size_t g = 0; g + 1 < c.gb.size(); ++g) {
        int o = 0;
        for (int l = c.gb[g]; l < c.gb[g + 1]; ++l)
            o += (log ? 2 : 1) * ((c.tx2 + 2 * (R[l] + (log ? 1 : 0)) + 3) & ~3);
        vrow = o > vrow ? o : vrow;
    }
    // mode 0: max/argmax ring, 1: response-stack ring, 2 (soft forward) and
    // 3 (level blur): none
    const int ring = c.rb + 2;
    const int ring_f = base == 0 ? ring * c.tx2 : base == 1 ? ring * layers * c.tx2 : 0;
    const int mask_bytes = layers > 32 ? 8 : 4;
    const int ring_b = base == 0   ? ((ring * c.tx2 + 15) & ~15)
                       : base == 1 ? ((ring * c.tx2 * mask_bytes + 15) & ~15)
                                   : 0;
    return 4 * (c.rb * vrow + ring_f) + ring_b + 4 * 64;
}

int wextp_of(const std::vector<int> &R, int mode, const TileConfig &c) {
    return (c.tx2 + 2 * halo_of(R, mode) + 3) & ~3;
}

}  // namespace

namespace {

// Tensor-core variant: the fp16 window (column groups of 8 columns, 16 bytes
// a row, groups padded so that four cover the 32 banks), the tap matrices
// (hi and lo parts per level group), the mbarrier / tensor-memory block.
int tc_window_bytes(const std::vector<int> &R, int mode, const TileConfig &c, int brows) {
    const int wext = c.tx2 + 2 * halo_of(R, mode);
    const int nmt = (wext + 127) / 128;
    const int gstr = ((16 * brows + 127) / 128) * 128 + 32;
    return nmt * 16 * gstr;
}

// K rows and N columns of group g's MMAs: the group's largest halo (R, or
// R + 1 for the LoG's second-difference taps) on both sides of the step's
// rows; rows x levels, twice for the LoG (g and g'' rows), padded to 16
void tc_group_dims(const std::vector<int> &R, int mode, const TileConfig &c, int g, int *kgp,
                   int *ngp) {
    const int extra = is_log(mode) ? 1 : 0;
    int rg = 0;
    for (int l = c.gb[g]; l < c.gb[g + 1]; ++l) rg = R[l] + extra > rg ? R[l] + extra : rg;
    *kgp = (c.rb + 2 * rg + 15) & ~15;
    *ngp = ((c.gb[g + 1] - c.gb[g]) * c.rb * (1 + extra) + 15) & ~15;
}

int tc_b_bytes(const std::vector<int> &R, int mode, const TileConfig &c) {
    int o = 0;
    for (size_t g = 0; g + 1 < c.gb.size(); ++g) {
        int kgp, ngp;
        tc_group_dims(R, mode, c, (int)g, &kgp, &ngp);
        o += 4 * kgp * ngp;
    }
    return o;
}

int tc_tmem_cols(const std::vector<int> &R, int mode, const TileConfig &c) {
    const int wext = c.tx2 + 2 * halo_of(R, mode);
    int nct = 0;
    for (size_t g = 0; g + 1 < c.gb.size(); ++g) {
        int kgp, ngp;
        tc_group_dims(R, mode, c, (int)g, &kgp, &ngp);
        nct += ngp;
    }
    return ((wext + 127) / 128) * nct;
}

int tc_min_rows(const std::vector<int> &R, int mode, const TileConfig &c) {
    return c.rb + 2 * halo_of(R, mode) + 2 * c.rb + 16;
}

}  // namespace

// Input window rows: one step's rows (rb + 2 rmax) plus up to four steps of
// slack (the window shifts back once the slack is used up), as many as fit.
// The tensor-core variant also holds the rows of the step after next and 16
// rows of K padding, and takes up to six steps of slack.
int brows_for(const std::vector<int> &R, int mode, const TileConfig &c) {
    if (c.tc == 2) return c.rb + 2 * halo_of(R, mode);  // the two-pass kernel has no row window
    if (c.tc) {
        const int lo = tc_min_rows(R, mode, c);
        const int fixed = smem_fixed(R, mode, c) + tc_b_bytes(R, mode, c) + 128;
        int b = lo + 6 * c.rb;
        while (b > lo && fixed + tc_window_bytes(R, mode, c, b) > kSmemLimit) --b;
        return b;
    }
    const int win = c.rb + 2 * halo_of(R, mode);
    const int row_bytes = 4 * wextp_of(R, mode, c);
    const int room = (kSmemLimit - smem_fixed(R, mode, c)) / row_bytes;
    int b = win + 4 * c.rb;
    if (b > room) b = room;
    return b < win ? win : b;
}

int smem_estimate(const std::vector<int> &R, int mode, const TileConfig &c) {
    if (c.tc == 2) return t2_smem(R, mode, c);
    if (c.tc)
        return smem_fixed(R, mode, c) + tc_b_bytes(R, mode, c) + 128 +
               tc_window_bytes(R, mode, c, brows_for(R, mode, c));
    return smem_fixed(R, mode, c) + 4 * brows_for(R, mode, c) * wextp_of(R, mode, c);
}

namespace {
double cost_model(const std::vector<int> &R, int mode, const TileConfig &c);
}

// Two-pass kernel (tc = 2): its shared memory as the kernel lays it out (the
// fp16 window with zero padding rows and columns for the K and N padding of
// every level's products, three tap-matrix buffers of hi and lo parts, the
// split V rows, the control block) and its tensor-memory columns (two V and
// two L buffers).
namespace {
struct T2Geom {
    int nvmax = 0, khmax = 0, smax = 0, xr = 0, xc = 0;
};
T2Geom t2_geom(const std::vector<int> &R, const TileConfig &c) {
    T2Geom g;
    const int rmax = rmax_of(R);
    auto c16 = [](int v) { return (v + 15) & ~15; };
    g.xr = 128 + 2 * rmax;
    int xc = c.tx2 + 2 * rmax;
    for (int r : R) {
        const int k0 = rmax - r, j0 = (rmax - r) & ~7, off = (rmax - r) & 7;
        const int need = c.tx2 + 2 * r;
        const int kv = c16(128 + 2 * r), nv = c16(off + need), kh = c16(need);
        g.nvmax = std::max(g.nvmax, nv);
        g.khmax = std::max(g.khmax, kh);
        g.smax = std::max(g.smax, kv / 8 + 15);
        g.xr = std::max(g.xr, k0 + kv);
        xc = std::max(xc, j0 + nv);
    }
    g.xc = (xc + 7) & ~7;
    return g;
}
}  // namespace

int t2_smem(const std::vector<int> &R, int mode, const TileConfig &c) {
    const T2Geom g = t2_geom(R, c);
    const int xgstr = ((16 * g.xr + 127) / 128) * 128 + 16;
    const int x_bytes = (g.xc / 8) * xgstr;
    const int tab_part = g.smax * 128;
    const int ah_part = 16 * (g.khmax / 8) * 128;
    int b = ((x_bytes + 127) & ~127) + 8 * tab_part + 2 * ah_part + 512 + 4 * ((g.xc + 3) & ~3);
    // 26-neighbour rule: two exchange buffers, the 16-bit layer masks
    const int cp = ((c.nt - 32) / 32) / 4;
    if (mode == MHFD_NMS_LOCAL26)
        b += 2 * 4 * (128 * cp * 2 + 8 * (c.tx2 + 4 * cp)) + 2 * c.tx2 * 128;
    return b;
}

// detection with the DoG response: the paper rule or the 26-neighbour rule
bool t2_mode_ok(int mode) { return mode == MHFD_NMS_PAPER || mode == MHFD_NMS_LOCAL26; }

bool t2_shape_ok(const std::vector<int> &R, int mode, const TileConfig &c, std::string *why) {
    auto no = [&](const char *m) {
        if (why) *why = m;
        return false;
    };
    if (!t2_mode_ok(mode)) return no("the two-pass kernel takes detection with the DoG response");
    if (mode == MHFD_NMS_LOCAL26 && R.size() - 1 > 16)
        return no("the two-pass kernel's 26-neighbour rule takes up to 16 layers");
    if (c.tx2 % 16 || c.tx2 < 16 || c.tx2 > 128)
        return no("the two-pass kernel's strips are 16 to 128 columns, a multiple of 16");
    if (c.ty2 != 128 || (c.nt != 288 && c.nt != 544))
        return no("the two-pass kernel: tiles of 128 rows, 288 or 544 threads");
    if (c.tx2 % (4 * ((c.nt - 32) / 128))) return no("the two-pass kernel: whole column parts of 4");
    const T2Geom g = t2_geom(R, c);
    if (g.nvmax > 256 || 2 * g.nvmax + 2 * c.tx2 > 512)
        return no("the two-pass kernel's V and L buffers exceed tensor memory for this ladder");
    if (8192 + 5 * c.tx2 * 128 > 2 * 16 * (g.khmax / 8) * 128)
        return no("the tile-end maxima test does not fit the split rows' space");
    if (t2_smem(R, mode, c) > kSmemLimitBytes) return no("does not fit in shared memory");
    return true;
}

TileConfig t2_config(int nl, int tx2) {
    TileConfig c;
    c.tx2 = tx2;
    c.ty2 = 128;
    c.rb = 4;
    c.nt = 288;
    c.gb = {0, nl};
    c.tc = 2;
    c.item = 1;
    return c;
}

// 64-column strips (62 x 126 outputs per tile: the per-thread responses of
// wider strips exceed the registers), else 48; a ladder whose halo leaves
// narrower strips only (tensor memory) takes the vertical-pass kernel, which
// wastes less on halos there
bool choose_tile_t2(const std::vector<int> &R, int mode, TileConfig *cfg, std::string *why) {
    for (int tx2 : {64, 48}) {
        const TileConfig c = t2_config((int)R.size(), tx2);
        if (t2_shape_ok(R, mode, c, why)) {
            *cfg = c;
            return true;
        }
    }
    return false;
}

// The vertical-pass kernel: the paper rule, DoG or LoG response; the
// 26-neighbour rule with the DoG response.  (With the scale-maximum masks and
// two-output items, the 26-neighbour rule runs faster on it at 160-wide
// strips, 2.23 ms, than on the FFMA kernel, 2.36 ms; its ring of all layers
// had left it 192-wide strips of one-row items, 5.5 ms.  The two-pass kernel
// takes the rule by default up to 16 layers, 0.85 ms.)
bool tc_mode_ok(int mode) { return (mode & 3) == 0 || mode == 1; }

bool tc_shape_ok(const std::vector<int> &R, int mode, const TileConfig &c, std::string *why) {
    auto no = [&](const char *m) {
        if (why) *why = m;
        return false;
    };
    if (!tc_mode_ok(mode)) return no("the tensor-core pass takes the DoG detection modes only");
    if (c.rb != 4 && c.rb != 8) return no("the tensor-core pass takes four or eight rows per step");
    if (c.nt % 32 || c.nt < 128 || c.nt > 1024) return no("threads: whole warps, at least one warpgroup");
    if (c.item < 1 || c.item > 3) return no("horizontal item kind 1, 2 or 3");
    if (h_items(c) > 2 * c.nt) return no("more than two horizontal items per thread");
    if (c.gb.size() - 1 > 12) return no("at most 12 level groups");
    if (tc_tmem_cols(R, mode, c) > 512) return no("tensor memory holds 512 columns");
    if (brows_for(R, mode, c) < tc_min_rows(R, mode, c) ||
        smem_estimate(R, mode, c) > kSmemLimit)
        return no("does not fit in shared memory");
    return true;
}

std::vector<TileConfig> tile_menu_tc(const std::vector<int> &R, int mode) {
    std::vector<TileConfig> out;
    if (!tc_mode_ok(mode)) return out;
    const int nl = (int)R.size();
    const int widths[] = {96, 128, 192, 224, 256, 288, 320, 352, 384, 448, 480, 512};
    const int threads[] = {128, 160, 192, 224, 256, 288, 384, 416, 512};
    // four rows per step on one-row items (eight rows of one-row items ran
    // at about twice the time on GB300: two items a thread on two warps per
    // scheduler); four or eight rows on two-row items (packed FMAs)
    for (int item : {1, 2, 3})
    for (int rb : {4, 8}) {
        if (item != 2 && rb == 8) continue;
        for (int tx2 : widths)
            for (int nt : threads) {
                const int items = (rb / (item == 2 ? 2 : 1)) * (tx2 / (item == 3 ? 2 : 4));
                if (items > 2 * nt || items <= nt - 128) continue;  // 1..2 items a thread, no idle warpgroup
                for (int ng = 1; ng <= 6 && ng <= nl; ++ng) {
                    TileConfig c;
                    c.tx2 = tx2;
                    c.ty2 = 2 + 16;
                    c.rb = rb;
                    c.nt = nt;
                    c.item = item;
                    c.gb.assign(ng + 1, 0);
                    for (int g = 0; g <= ng; ++g) c.gb[g] = (int)((long long)nl * g / ng);
                    c.tc = 1;
                    if (tc_shape_ok(R, mode, c, nullptr)) out.push_back(c);
                }
            }
    }
    return out;
}

// The FFMA kernel sharing a tensor-core shape's tile grid (strip width and
// tile height): four (else two) rows per step, a thread per halo'd column
// and per horizontal item, the fewest level groups that fit, then the cost
// model.
bool companion_tile(const std::vector<int> &R, int mode, const TileConfig &tc, TileConfig *cfg) {
    const int nl = (int)R.size();
    const int wext = tc.tx2 + 2 * halo_of(R, mode);
    bool found = false;
    double best = 0.0;
    for (int rb : {4, 2}) {
        const int items = rb * (tc.tx2 / 4);
        int nt = wext > items ? wext : items;
        nt = (nt + 31) / 32 * 32;
        if (nt > 1024) nt = ((items + 31) / 32) * 32;
        for (int ng = 1; ng <= 12 && ng <= nl; ++ng) {
            TileConfig c;
            c.tx2 = tc.tx2;
            c.ty2 = tc.ty2;
            c.rb = rb;
            c.nt = nt;
            c.gb.assign(ng + 1, 0);
            for (int g = 0; g <= ng; ++g) c.gb[g] = (int)((long long)nl * g / ng);
            if (smem_estimate(R, mode, c) > kSmemLimit) continue;
            const double cost = cost_model(R, mode, c);
            if (!found || cost < best) {
                best = cost;
                *cfg = c;
                found = true;
            }
        }
        if (found) return true;
    }
    return false;
}

// Widest strip whose horizontal items leave exactly one warp free for the
// MMA issue (tx2 = threads - 32, one item per thread: the four schedulers
// then hold equal work), fewest groups.
bool choose_tile_tc(const std::vector<int> &R, int mode, TileConfig *cfg, std::string *why) {
    const std::vector<TileConfig> menu = tile_menu_tc(R, mode);
    bool found = false;
    TileConfig comp;
    for (const TileConfig &c : menu) {
        if (c.rb != 4 || c.item != 1 || c.tx2 != c.nt - 32 || c.nt * 168 > 65536 ||
            !companion_tile(R, mode, c, &comp))
            continue;
        if (!found || c.tx2 > cfg->tx2 ||
            (c.tx2 == cfg->tx2 && c.gb.size() < cfg->gb.size())) {
            *cfg = c;
            found = true;
        }
    }
    for (const TileConfig &c : menu) {
        if (found) break;
        if (companion_tile(R, mode, c, &comp)) {
            *cfg = c;
            found = true;
        }
    }
    if (!found && why) *why = "no tensor-core tile configuration fits for this ladder";
    return found;
}

namespace {

std::vector<int> groups_for(int nl, int max_per_group) {
    const int ng = (nl + max_per_group - 1) / max_per_group;
    std::vector<int> gb(ng + 1);
    for (int g = 0; g <= ng; ++g) gb[g] = (int)((long long)nl * g / ng);
    return gb;
}

// relative instruction cost per output pixel (FMA-dominated model): the
// vertical pass over each group's halo'd columns (a group needing more than
// one round of nt threads is charged for the idle thread slots of its last
// round, which wait at the next barrier), the horizontal pass over the
// strip's columns, and the window shifts
double cost_model(const std::vector<int> &R, int mode, const TileConfig &c) {
    const int rmax = halo_of(R, mode);
    const double tx = c.tx2 - 2;
    double v = 0, h = 0;
    for (size_t g = 0; g + 1 < c.gb.size(); ++g) {
        int rg = 0;
        double w = 0;
        for (int l = c.gb[g]; l < c.gb[g + 1]; ++l) {
            rg = R[l] > rg ? R[l] : rg;
            w += R[l] + 1;
        }
        w += rg;  // folded sums of the group
        const int cols = c.tx2 + 2 * rg;
        const double slots = cols <= c.nt ? cols : ((cols + c.nt - 1) / c.nt) * (double)c.nt;
        v += w * slots / tx;
    }
    for (int r : R) h += 2 * r + 1;
    const double h_eff = h * (c.tx2 / tx);
    const int brows = brows_for(R, mode, c);
    const int steps_per_shift = (brows - (c.rb + 2 * rmax)) / c.rb + 1;
    const double wext = c.tx2 + 2 * rmax;
    const double shift = 4.0 * 2 * rmax * wext / (steps_per_shift * c.rb * tx);
    return v + h_eff + shift;
}

}  // namespace

std::vector<TileConfig> tile_menu(const std::vector<int> &R, int mode) {
    std::vector<TileConfig> out;
    const int nl = (int)R.size();
    const int rmax = halo_of(R, mode);
    const int widths[] = {64, 96, 128, 160, 192, 224, 256, 288, 320};
    const int gmax[] = {6, 8, 10, 12};
    for (int tx2 : widths) {
        const int wext = tx2 + 2 * rmax;
        for (int nt = 64; nt <= 512; nt += 32) {
            if (nt < wext / 3) continue;
            const int rb_full = nt / (tx2 / 4);  // horizontal items == threads
            for (int rb = 2; rb <= 12; ++rb) {
                if (rb != rb_full && rb != rb_full / 2 && rb != 4 && rb != 8) continue;
                for (int gm : gmax) {
                    TileConfig c;
                    c.tx2 = tx2;
                    c.nt = nt;
                    c.rb = rb;
                    c.gb = groups_for(nl, gm);
                    c.ty2 = 2 + 16;  // tiles of 16 output rows
                    if (smem_estimate(R, mode, c) > kSmemLimit) continue;
                    out.push_back(c);
                }
            }
        }
    }
    return out;
}

bool choose_tile(const std::vector<int> &R, int mode, TileConfig *cfg, std::string *why) {
    const std::vector<TileConfig> menu = tile_menu(R, mode);
    const int rmax = halo_of(R, mode);
    // Preferred shapes (what the autotuner finds on GB300): four rows per
    // step (one vertical part, enough rows to amortise a step's barriers and
    // scans), one thread per halo'd column so that the vertical pass of every
    // group is a single round, at most 512 threads (at least 128 registers
    // each), every horizontal item with a thread.  Among them, and failing
    // that among all balanced shapes, the cost model decides.
    for (int pass = 0; pass < 2; ++pass) {
        double best = 1e300;
        bool found = false;
        for (const TileConfig &c : menu) {
            const int wext = c.tx2 + 2 * rmax;
            const int ncol = (wext + 31) / 32 * 32;
            if (c.rb * (c.tx2 / 4) > c.nt) continue;
            if (pass == 0 && (c.rb != 4 || c.nt < ncol || c.nt > ncol + 32 || c.nt > 512))
                continue;
            if (pass == 1 && (c.nt < wext - 31 || c.nt > wext + 31)) continue;
            const double cost = cost_model(R, mode, c);
            if (cost < best) {
                best = cost;
                *cfg = c;
                found = true;
            }
        }
        if (found) return true;
    }
    if (why) *why = "no tile configuration fits in shared memory for this ladder";
    return false;
}

namespace {
std::string source_hash(const std::string &src) {
    std::string opts;
    for (const char *o : kOpts) opts += std::string(o) + " ";
    int ver_major = 0, ver_minor = 0;
    nvrtcVersion(&ver_major, &ver_minor);
    char hbuf[32];
    std::snprintf(hbuf, sizeof(hbuf), "%016llx",
                  fnv1a(src + opts + std::to_string(ver_major) + "." + std::to_string(ver_minor)));
    return hbuf;
}
}  // namespace

int precompile_variant(const LadderKey &lk, int mode, int store, const TileConfig &cfg) {
    if (smem_estimate(lk.R, mode | (lk.response ? kModeLog : 0), cfg) > kSmemLimit)
        return fail(MHFD_ERR_UNSUPPORTED, "tile configuration exceeds shared memory");
    const std::string src = make_source(lk, mode, store, cfg);
    const std::string path = cache_dir() + "/" + source_hash(src) + ".cubin";
    std::string cubin;
    if (read_file(path, &cubin)) return MHFD_OK;
    const int rc = compile_cubin(src, &cubin);
    if (rc != MHFD_OK) return rc;
    write_file_atomic(path, cubin);
    return MHFD_OK;
}

int get_variant(const LadderKey &lk, int mode, int store, const TileConfig &cfg, Variant **out) {
    const std::vector<int> &R = lk.R;
    int dev = 0;
    MHFD_CUDA(cudaGetDevice(&dev));
    MHFD_CUDA(cudaFree(nullptr));  // make sure the primary context exists and is current
    const std::string src = make_source(lk, mode, store, cfg);
    const std::string hbuf = source_hash(src);
    const std::string key = hbuf + "@" + std::to_string(dev);
    {
        std::lock_guard<std::mutex> guard(g_mu);
        auto it = g_variants.find(key);
        if (it != g_variants.end()) {
            *out = it->second;
            return MHFD_OK;
        }
    }
    if (smem_estimate(R, mode | (lk.response ? kModeLog : 0), cfg) > kSmemLimit)
        return fail(MHFD_ERR_UNSUPPORTED, "tile configuration exceeds shared memory");
    const std::string path = cache_dir() + "/" + hbuf + ".cubin";
    std::string cubin;
    if (!read_file(path, &cubin)) {
        const int rc = compile_cubin(src, &cubin);
        if (rc != MHFD_OK) return rc;
        write_file_atomic(path, cubin);
    }
    if (!drv().ok) return fail(MHFD_ERR_CUDA, "CUDA driver entry points unavailable");
    Variant *v = new Variant();
    v->key = key;
    v->cfg = cfg;
    CUresult r = drv().moduleLoadData(&v->mod, cubin.data());
    if (r != CUDA_SUCCESS) {
        delete v;
        return drv_fail(r, "cuModuleLoadData");
    }
    r = drv().moduleGetFunction(&v->fn, v->mod, "mhfd_fused_detect");
    if (r != CUDA_SUCCESS) return drv_fail(r, "cuModuleGetFunction");
    CUdeviceptr gp;
    size_t gsz;
    int vals[3] = {0, 0, 0};
    const char *names[3] = {"mhfd_smem_bytes", "mhfd_param_bytes", "mhfd_ntaps"};
    for (int i = 0; i < 3; ++i) {
        r = drv().moduleGetGlobal(&gp, &gsz, v->mod, names[i]);
        if (r != CUDA_SUCCESS) return drv_fail(r, "cuModuleGetGlobal");
        r = drv().memcpyDtoH(&vals[i], gp, sizeof(int));
        if (r != CUDA_SUCCESS) return drv_fail(r, "cuMemcpyDtoH");
    }
    v->smem_bytes = vals[0];
    v->param_bytes = vals[1];
    v->ntaps = vals[2];
    if (v->smem_bytes > kSmemLimit) return fail(MHFD_ERR_UNSUPPORTED, "kernel shared memory too large");
    r = drv().funcSetAttribute(v->fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, v->smem_bytes);
    if (r != CUDA_SUCCESS) return drv_fail(r, "cuFuncSetAttribute");
    r = drv().occupancy(&v->occupancy, v->fn, cfg.nt, (size_t)v->smem_bytes);
    if (r != CUDA_SUCCESS) return drv_fail(r, "cuOccupancyMaxActiveBlocksPerMultiprocessor");
    if (v->occupancy < 1) return fail(MHFD_ERR_UNSUPPORTED, "fused kernel does not fit on an SM");
    if (cfg.tc == 2) {
        // the two-pass kernel copies each level's tap matrices from global
        // memory: build them once, here (the module's setup kernel)
        CUfunction fset;
        r = drv().moduleGetFunction(&fset, v->mod, "mhfd_t2_tables");
        if (r != CUDA_SUCCESS) return drv_fail(r, "cuModuleGetFunction");
        int tab_bytes = 0;
        r = drv().moduleGetGlobal(&gp, &gsz, v->mod, "mhfd_t2_tab_bytes");
        if (r != CUDA_SUCCESS) return drv_fail(r, "cuModuleGetGlobal");
        r = drv().memcpyDtoH(&tab_bytes, gp, sizeof(int));
        if (r != CUDA_SUCCESS) return drv_fail(r, "cuMemcpyDtoH");
        cudaError_t e = cudaMalloc(&v->t2tab, (size_t)tab_bytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (tap matrices)");
        void *targ = v->t2tab;
        void *args[] = {&targ};
        r = drv().launchKernel(fset, (unsigned)R.size(), 1, 1, (unsigned)(cfg.nt - 32), 1, 1, 0, nullptr,
                               args, nullptr);
        if (r != CUDA_SUCCESS) return drv_fail(r, "cuLaunchKernel (tap matrices)");
        e = cudaStreamSynchronize(nullptr);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize (tap matrices)");
    }
    std::lock_guard<std::mutex> guard(g_mu);
    auto it = g_variants.find(key);
    if (it != g_variants.end()) {  // another thread won the race
        if (v->t2tab) cudaFree(v->t2tab);
        drv().moduleUnload(v->mod);
        delete v;
        *out = it->second;
        return MHFD_OK;
    }
    g_variants[key] = v;
    *out = v;
    return MHFD_OK;
}

}  // namespace mhfd
