// Run-time specialised tile passes and whole-row kernels.
//
// The forward tile kernel interprets each pass's op program from shared
// memory: per op it reads the decoded record, dispatches on its handler and
// forms control masks at run time.  For a circuit that runs many times the
// same passes can be compiled instead: this file writes, for every pass of a
// schedule, an op runner whose body is the pass's ops as direct calls into
// the engine's handlers (dq_engine.cuh) with every register position,
// control mask, lane bit and layout as a literal, instantiates the shared
// kernel body (dq_tile_fwd.cuh) with it, compiles all passes of the schedule
// in one NVRTC program for the device's architecture and loads the result
// with the runtime's library API.  The arithmetic per element is the
// interpreter's; only the dispatch is gone.  Reverse-sweep tile passes
// (dq_tile_adj.cuh) and the whole-row kernel (dq_rows_body.cuh, one kernel
// per circuit program) are specialised the same way.  NVRTC is opened with
// dlopen on first use: without it the interpreter simply stays in use.
#include <dlfcn.h>
#include <nvrtc.h>
#include <sys/stat.h>
#include <unistd.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <sstream>
#include <string>
#include <thread>
#include <vector>
#include <algorithm>

#include "dq_jit.h"
#include "dq_rows.h"
#include "dq_tile.h"
#include "jit_headers.inc"   // generated by build.py: the device headers' texts

namespace dq {

namespace {

struct NvrtcApi {
    bool ok = false;
    nvrtcResult (*create)(nvrtcProgram *, const char *, const char *, int, const char *const *,
                          const char *const *) = nullptr;
    nvrtcResult (*compile)(nvrtcProgram, int, const char *const *) = nullptr;
    nvrtcResult (*log_size)(nvrtcProgram, size_t *) = nullptr;
    nvrtcResult (*log)(nvrtcProgram, char *) = nullptr;
    nvrtcResult (*cubin_size)(nvrtcProgram, size_t *) = nullptr;
    nvrtcResult (*cubin)(nvrtcProgram, char *) = nullptr;
    nvrtcResult (*destroy)(nvrtcProgram *) = nullptr;
    nvrtcResult (*version)(int *, int *) = nullptr;
};

NvrtcApi &nvrtc_api() {
    static NvrtcApi api;
    static std::once_flag once;
    std::call_once(once, [] {
        void *h = nullptr;
        for (const char *name : {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13"}) {
            h = dlopen(name, RTLD_NOW | RTLD_LOCAL);
            if (h) break;
        }
        if (!h) return;
        api.create = reinterpret_cast<decltype(api.create)>(dlsym(h, "nvrtcCreateProgram"));
        api.compile = reinterpret_cast<decltype(api.compile)>(dlsym(h, "nvrtcCompileProgram"));
        api.log_size = reinterpret_cast<decltype(api.log_size)>(dlsym(h, "nvrtcGetProgramLogSize"));
        api.log = reinterpret_cast<decltype(api.log)>(dlsym(h, "nvrtcGetProgramLog"));
        api.cubin_size = reinterpret_cast<decltype(api.cubin_size)>(dlsym(h, "nvrtcGetCUBINSize"));
        api.cubin = reinterpret_cast<decltype(api.cubin)>(dlsym(h, "nvrtcGetCUBIN"));
        api.destroy = reinterpret_cast<decltype(api.destroy)>(dlsym(h, "nvrtcDestroyProgram"));
        api.version = reinterpret_cast<decltype(api.version)>(dlsym(h, "nvrtcVersion"));
        api.ok = api.create && api.compile && api.log_size && api.log && api.cubin_size && api.cubin && api.destroy;
    });
    return api;
}

// ---- compiled-program cache -------------------------------------------------
// A compiled program is kept on disk under a key of everything that decides
// its bytes: the generated source, the target architecture, the embedded
// device headers and the NVRTC version.  The folder is DQ_JIT_CACHE when set
// (empty or "0": no cache), else _jit_cache next to this library.
uint64_t fnv64(uint64_t h, const void *p, size_t n) {
    const unsigned char *b = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
    return h;
}

std::string cache_dir() {
    if (const char *env = std::getenv("DQ_JIT_CACHE")) {
        if (!*env || std::strcmp(env, "0") == 0) return std::string();
        return env;
    }
    Dl_info info;
    if (!dladdr(reinterpret_cast<void *>(&cache_dir), &info) || !info.dli_fname) return std::string();
    std::string lib = info.dli_fname;
    const size_t slash = lib.rfind('/');
    return (slash == std::string::npos ? std::string(".") : lib.substr(0, slash)) + "/_jit_cache";
}

std::string cache_path(const std::string &src, int cc) {
    const std::string dir = cache_dir();
    if (dir.empty()) return std::string();
    int major = 0, minor = 0;
    if (nvrtc_api().version) nvrtc_api().version(&major, &minor);
    uint64_t h1 = 1469598103934665603ull, h2 = 7809847782465536322ull;
    auto mix = [&](const void *p, size_t n) {
        h1 = fnv64(h1, p, n);
        h2 = fnv64(h2 ^ 0x9e3779b97f4a7c15ull, p, n);
    };
    mix(src.data(), src.size());
    const int meta[3] = {cc, major, minor};
    mix(meta, sizeof(meta));
    for (int i = 0; i < kJitHeaderCount; ++i) mix(kJitHeaderTexts[i], std::strlen(kJitHeaderTexts[i]));
    char name[64];
    std::snprintf(name, sizeof(name), "/%016llx%016llx.cubin", (unsigned long long)h1, (unsigned long long)h2);
    return dir + name;
}

bool cache_read(const std::string &path, std::vector<char> *cubin) {
    FILE *f = path.empty() ? nullptr : std::fopen(path.c_str(), "rb");
    if (!f) return false;
    std::vector<char> buf;
    char chunk[65536];
    size_t got;
    while ((got = std::fread(chunk, 1, sizeof(chunk), f)) > 0) buf.insert(buf.end(), chunk, chunk + got);
    std::fclose(f);
    if (buf.size() < 4 || std::memcmp(buf.data(), "\x7f" "ELF", 4) != 0) return false;   // not a cubin
    cubin->swap(buf);
    return true;
}

void cache_write(const std::string &path, const std::vector<char> &cubin) {
    if (path.empty()) return;
    const std::string dir = path.substr(0, path.rfind('/'));
    mkdir(dir.c_str(), 0755);   // may exist
    const std::string tmp = path + ".tmp" + std::to_string((long long)getpid());
    FILE *f = std::fopen(tmp.c_str(), "wb");
    if (!f) return;
    const bool ok = std::fwrite(cubin.data(), 1, cubin.size(), f) == cubin.size();
    std::fclose(f);
    if (!ok || std::rename(tmp.c_str(), path.c_str()) != 0) std::remove(tmp.c_str());
}

std::string hex32(uint32_t v) {
    char b[16];
    std::snprintf(b, sizeof(b), "0x%08xu", v);
    return b;
}

// The control mask expression of an op in its layout (the interpreter's
// op_cmask with the mode resolved).
std::string cmask_expr(const EOp &o) {
    if (o.cmode == 0) return hex32(o.cmc);
    if (o.cmode == 1) return "(((L.tb >> " + std::to_string((int)o.carg) + ") & 1u) ? ~0u : 0u)";
    return "(((base >> " + std::to_string((int)o.carg) + ") & 1ull) ? ~0u : 0u)";
}

// An EOp literal (variable `v`) for the handlers that read its fields.
std::string eop_literal(const EOp &o, const char *v = "o") {
    std::ostringstream s;
    s << "EOp " << v << "{}; " << v << ".h = " << o.h << "; " << v << ".kind = " << o.kind << "; " << v
      << ".cmc = " << hex32(o.cmc) << "; " << v << ".cmode = " << (int)o.cmode << "; " << v
      << ".carg = " << (int)o.carg << "; " << v << ".tmode = " << (int)o.tmode << "; " << v
      << ".targ = " << (int)o.targ << "; " << v << ".slot = " << o.slot << ";";
    return s.str();
}

// Gradient partial of an op with a local slot into the per-warp accumulators.
void emit_acc(std::ostringstream &s, const char *g, int slot, int nslot) {
    if (slot < 0) return;
    s << " { const R gs = warp_sum_t(" << g << "); if (lane == 0) accw[warp * " << nslot << " + " << slot
      << "] += gs; }";
}

// One reverse op (coefficient scoef[i]) as a direct call of its adjoint
// handler: eng_adjoint's dispatch resolved here, with the gradient partial
// formed only for an op with a slot (added to accw[warp * nacc + slot]).
// pd: parity-diagonal ops have their own handler (else they take the
// uniform-diagonal one, as in a kernel compiled without them).
void emit_adj_op(std::ostringstream &s, const EOp &o, int i, int M, bool pd, int nacc) {
    const int h = o.h;
    const char *G = o.slot >= 0 ? "true" : "false";
    const std::string ud = "const Mat2<R> ud = dagger(scoef[" + std::to_string(i) + "]);";
    std::string body;
    if (h < H_GEN || (h >= H_DIAG && h < H_CREAL)) {
        const int P = h < H_GEN ? h - H_REAL : h - H_DIAG;
        if (P >= M) return;
        if (h < H_GEN)
            body = std::string("gv = adj_pairs_at<R, M, ") + std::to_string(P) + ", CLS_REAL, " + G + ">(ps, ls, ud);";
        else
            body = std::string("gv = adj_diag_at<R, M, ") + std::to_string(P) + ", " + G + ">(ps, ls, ud, " +
                   std::to_string((int)o.kind) + ");";
    } else if (pd && h == H_PDIAG) {
        body = eop_literal(o) + std::string(" gv = adj_pdiag<R, M, ") + G + ">(ps, ls, o, ud, base, L);";
    } else {
        if (o.cmode == 0 && o.cmc == 0) return;   // the control is never set in this layout
        std::string call;
        auto reg = [&](int base_h, const char *tmpl, const char *cls, const char *g, bool kind) {
            const int P = h - base_h;
            if (P >= M) return false;
            call = std::string(tmpl) + "<R, M, " + std::to_string(P) + (cls ? std::string(", ") + cls : "") + ", " +
                   g + ">(ps, ls, ud, " + (kind ? std::to_string((int)o.kind) + ", " : "") + "cm)";
            return true;
        };
        bool ok = true;
        if (h >= H_GEN && h < H_ANTI) ok = reg(H_GEN, "adj_pairs_sel", "CLS_GENERAL", G, false);
        else if (h >= H_ANTI && h < H_DIAG) ok = reg(H_ANTI, "adj_pairs_sel", "CLS_ANTI", "false", false);
        else if (h >= H_CREAL && h < H_CDIAG) ok = reg(H_CREAL, "adj_pairs_sel", "CLS_REAL", G, false);
        else if (h >= H_CDIAG && h < H_LREAL) ok = reg(H_CDIAG, "adj_diag_sel", nullptr, G, true);
        else if (h == H_LREAL || h == H_LGEN || h == H_LANTI)
            call = std::string("adj_lane_at<R, M, ") +
                   (h == H_LREAL ? "CLS_REAL" : h == H_LGEN ? "CLS_GENERAL" : "CLS_ANTI") + ", " +
                   (h == H_LANTI ? "false" : G) + ">(ps, ls, ud, " + std::to_string((int)o.targ) + ", lane, cm)";
        else
            call = eop_literal(o) + std::string(" gv = adj_diag_uni<R, M, ") + G + ">(ps, ls, ud, o, L, base, cm)";
        if (!ok) return;
        body = "const uint32_t cm = " + cmask_expr(o) + ";";
        if (o.cmode != 0) body += " if (!__all_sync(0xffffffffu, cm == 0u))";
        if (call.compare(0, 4, "EOp ") == 0) {
            // the literal precedes the call inside its own block
            const size_t at = call.find(" gv = ");
            body = call.substr(0, at) + " " + body + " " + call.substr(at + 1) + ";";
        } else {
            body += " gv = " + call + ";";
        }
    }
    s << "        { " << ud << " R gv = R(0); " << body;
    emit_acc(s, "gv", o.slot, nacc);
    s << " }\n";
}

// A rotation pair in the reverse sweep: the DIAG op d (coefficient
// scoef[i]) and the REAL op r before it (scoef[i - 1]) un-applied in one
// register sweep (eng_adjoint_pair's dispatch resolved here).
void emit_adj_pair(std::ostringstream &s, const EOp &d, const EOp &r, int i, int M, int nacc) {
    const char *G = (d.slot >= 0 || r.slot >= 0) ? "true" : "false";
    std::string call;
    if (r.h == H_LREAL) {
        call = std::string("adj_pair_lane<R, M, ") + G + ">(ps, ls, dd, rr, " + std::to_string((int)d.kind) + ", " +
               std::to_string((int)r.targ) + ", lane, gd, gr);";
    } else {
        const int P = r.h - H_REAL;
        if (P >= 0 && P < 5 && P < M)
            call = std::string("adj_pair_reg<R, M, ") + std::to_string(P) + ", " + G + ">(ps, ls, dd, rr, " +
                   std::to_string((int)d.kind) + ", gd, gr);";
    }
    s << "        { const Mat2<R> dd = dagger(scoef[" << i << "]), rr = dagger(scoef[" << i - 1
      << "]); R gd = R(0), gr = R(0); " << call;
    emit_acc(s, "gd", d.slot, nacc);
    emit_acc(s, "gr", r.slot, nacc);
    s << " }\n";
}

// One reverse segment of a pass: gradient partials and un-application of
// its ops, highest first (a rotation pair consumes its REAL op too).
void emit_rev_segment(std::ostringstream &s, const TileSchedule &sc, const TPass &ps, const TSeg &sg, bool last) {
    const int M = sc.M;
    s << "    {\n        ESeg sg{}; ";
    for (int b = 0; b < M; ++b) s << "sg.B[" << b << "] = " << (int)sg.B[b] << "; ";
    s << "\n        const Layout L = make_layout(sg, M, " << sc.k << ", lane, warp);\n"
         "        eng_load<R, M>(ps, bufP, L);\n        eng_load<R, M>(ls, bufL, L);\n";
    if (last) s << "        io.prefetch();\n";
    for (int cc = 0; cc < sg.nops; ++cc) {
        const int oi = sg.op0 - ps.op0 - cc;
        const EOp &o = sc.rops[ps.op0 + oi];
        if (o.pad[1]) {
            emit_adj_pair(s, o, sc.rops[ps.op0 + oi - 1], oi, M, ps.nslot);
            ++cc;
            continue;
        }
        emit_adj_op(s, o, oi, M, false, ps.nslot);
    }
    if (last)
        s << "        io.template store<M>(ps, ls, L);\n    }\n";
    else
        s << "        eng_store<R, M>(ps, bufP, L);\n        eng_store<R, M>(ls, bufL, L);\n        __syncthreads();\n"
             "    }\n";
}

// One op of a pass (index i in the pass's op list); returns the number of
// ops it stands for (a controlled-phase fan consumes its members).
int emit_op(std::ostringstream &s, const EOp *ops, int i, int nops, bool pd) {
    const EOp &o = ops[i];
    const std::string u = "scoef[" + std::to_string(i) + "]";
    const int h = o.h;
    if (h < H_GEN) {
        s << "        pairs_at<R, M, " << h - H_REAL << ", CLS_REAL>(r, " << u << ");\n";
        return 1;
    }
    if (h >= H_DIAG && h < H_CREAL) {
        s << "        diag_at<R, M, " << h - H_DIAG << ">(r, " << u << ");\n";
        return 1;
    }
    if (h == H_PDIAG) {
        if (pd) s << "        { " << eop_literal(o) << " eng_pdiag<R, M>(r, o, " << u << ", base, L); }\n";
        return 1;
    }
    if (h == H_FAN) {
        s << "        eng_fan<R, M>(r, sops + " << i << ", scoef + " << i << ", base, L);\n";
        return std::max(1, (int)o.pad[0]);
    }
    if (h >= H_FAN) return 1;   // a fan member outside its fan (not produced by the planner)
    if (o.cmode == 0 && o.cmc == 0) return 1;   // the control is never set in this layout
    std::string call;
    if (h >= H_GEN && h < H_ANTI)
        call = "pairs_sel<R, M, " + std::to_string(h - H_GEN) + ", CLS_GENERAL>(r, " + u + ", cm)";
    else if (h >= H_ANTI && h < H_DIAG)
        call = "pairs_sel<R, M, " + std::to_string(h - H_ANTI) + ", CLS_ANTI>(r, " + u + ", cm)";
    else if (h >= H_CREAL && h < H_CDIAG)
        call = "pairs_sel<R, M, " + std::to_string(h - H_CREAL) + ", CLS_REAL>(r, " + u + ", cm)";
    else if (h >= H_CDIAG && h < H_LREAL)
        call = "diag_sel<R, M, " + std::to_string(h - H_CDIAG) + ">(r, " + u + ", cm)";
    else if (h == H_LREAL || h == H_LGEN || h == H_LANTI)
        call = std::string("lane_at<R, M, ") + (h == H_LREAL ? "CLS_REAL" : h == H_LGEN ? "CLS_GENERAL" : "CLS_ANTI") +
               ">(r, " + u + ", " + std::to_string((int)o.targ) + ", lane, cm)";
    else
        call = "diag_uni<R, M>(r, " + u + ", o, L, base, cm)";
    s << "        { const uint32_t cm = " << cmask_expr(o) << ";";
    if (h == H_DUNI) s << " " << eop_literal(o);
    if (o.cmode != 0) s << " if (!__all_sync(0xffffffffu, cm == 0u))";
    s << " " << call << "; }\n";
    return 1;
}

// Fixed-width integer names for the device headers (NVRTC has no libc).
const char *const kPrelude =
    "typedef signed char int8_t; typedef unsigned char uint8_t; typedef short int16_t;\n"
    "typedef unsigned short uint16_t; typedef int int32_t; typedef unsigned int uint32_t;\n"
    "typedef long long int64_t; typedef unsigned long long uint64_t; typedef unsigned long long uintptr_t;\n";

// Register-layout literal of a segment and the layout it makes.
void emit_layout(std::ostringstream &s, const ESeg &sg, int M, int n, const char *assign) {
    s << "        { ESeg sg{}; ";
    for (int b = 0; b < M; ++b) s << "sg.B[" << b << "] = " << (int)sg.B[b] << "; ";
    s << assign << "make_layout(sg, M, " << n << ", lane, warp); }\n";
}

// Whole-row reverse sweep: segments from the last op down (the first one in
// the layout lambda was formed in), each op's gradient partial added to its
// accumulator (stride nacc per warp); the sweep ends after `nrun` segments.
void emit_rows_reverse(std::ostringstream &s, const RowProgram &rp, int nacc) {
    for (size_t si = 0; si < rp.rsegs.size(); ++si) {
        const ESeg &sg = rp.rsegs[si];
        if (si > 0) {
            s << "        if (nrun <= " << si << ") return;\n"
                 "        eng_store<R, M>(ps, bufP, L);\n        eng_store<R, M>(ls, bufL, L);\n"
                 "        __syncthreads();\n";
            emit_layout(s, sg, rp.M, rp.n, "L = ");
            s << "        eng_load<R, M>(ps, bufP, L);\n        eng_load<R, M>(ls, bufL, L);\n";
        }
        for (int c = 0; c < sg.nops; ++c) {
            const int oi = sg.op0 - c;
            const EOp &o = rp.rops[oi];
            if (o.pad[1]) {
                emit_adj_pair(s, o, rp.rops[oi - 1], oi, rp.M, nacc);
                ++c;
                continue;
            }
            emit_adj_op(s, o, oi, rp.M, rp.pdiag, nacc);
        }
    }
}

}  // namespace

// Source of the whole-row kernel with the program's ops compiled in: one op
// runner (forward segments; reverse segments with gradient partials) and the
// kernel dq_jit_rows.
std::string jit_rows_source(const RowProgram &rp, int amp, int rpc) {
    const char *R = amp == 16 ? "double" : "float";
    const int M = rp.M;
    const int maxt = (((1 << M) * amp <= 64) ? 512 : 256) * rpc;
    const int minb = (amp == 8 && rpc == 1) ? 2 : 1;
    const int nacc = rp.nacc_shared + rp.nacc_row;
    std::ostringstream s;
    s << kPrelude << "#include \"dq_rows_body.cuh\"\nnamespace dq {\nnamespace {\n"
         "struct JitRows {\n"
         "    template <typename R, int M, bool PD>\n"
         "    __device__ __forceinline__ static void fwd(cx<R> (&r)[1 << M], cx<R> *bufP, Layout &L, const ESeg *,\n"
         "        const EOp *sops, const Mat2<R> *scoef, int, int, int lane, int warp) {\n"
         "        const uint64_t base = 0;\n";
    for (size_t si = 0; si < rp.fsegs.size(); ++si) {
        const ESeg &sg = rp.fsegs[si];
        if (si > 0) {
            s << "        eng_store<R, M>(r, bufP, L);\n        __syncthreads();\n";
            emit_layout(s, sg, M, rp.n, "L = ");
            s << "        eng_load<R, M>(r, bufP, L);\n";
        }
        for (int i = sg.op0; i < sg.op0 + sg.nops;) i += emit_op(s, rp.fops.data(), i, (int)rp.fops.size(), rp.pdiag);
    }
    s << "    }\n"
         "    template <typename R, int M, bool PD>\n"
         "    __device__ __forceinline__ static void rev(cx<R> (&ps)[1 << M], cx<R> (&ls)[1 << M], cx<R> *bufP,\n"
         "        cx<R> *bufL, Layout &L, const ESeg *, const EOp *, const Mat2<R> *scoef, R *accw, int, int nrun,\n"
         "        int, int lane, int warp) {\n"
         "        const uint64_t base = 0;\n";
    emit_rows_reverse(s, rp, nacc);
    s << "    }\n};\n}  // namespace\n}  // namespace dq\n"
      << "extern \"C\" __global__ void __launch_bounds__(" << maxt << ", " << minb << ") dq_jit_rows(dq::RowArgs a) {\n"
      << "    dq::rows_body<" << R << ", " << M << ", " << (rp.pdiag ? "true" : "false") << ", dq::JitRows, " << rpc
      << ">(a);\n}\n";
    return s.str();
}

// Source of passes [p0, p1) of the schedule (all when p1 < 0): op runner +
// kernel per pass.
std::string jit_source(const TileSchedule &sc, int amp, std::vector<std::string> &names, int p0, int p1) {
    if (p1 < 0) p1 = (int)sc.passes.size();
    const char *R = amp == 16 ? "double" : "float";
    const int M = sc.M;
    const int cxb = amp;   // bytes of one amplitude
    const int maxt = ((1 << M) * cxb >= 256) ? 256 : 512;
    const int minb = ((1 << M) * cxb <= 64) ? 2 : 1;
    std::ostringstream s;
    s << kPrelude;
    if (sc.adjoint) {
        // reverse passes: runner + kernel per pass
        const int amax = ((1 << M) * cxb <= 64) ? 512 : 256;
        s << "#include \"dq_tile_adj.cuh\"\nnamespace dq {\nnamespace {\n";
        for (int p = p0; p < p1; ++p) {
            const TPass &ps = sc.passes[p];
            s << "struct JitRev" << p << " {\n"
                 "    template <typename R, int M>\n"
                 "    __device__ __forceinline__ static void run(cx<R> (&ps)[1 << M], cx<R> (&ls)[1 << M],\n"
                 "        cx<R> *bufP, cx<R> *bufL, const EOp *, const ESeg *, const Mat2<R> *scoef, R *accw,\n"
                 "        int, int, int, int, uint64_t base, int lane, int warp, const AdjIo<R> &io) {\n";
            if (ps.nrseg == 0) s << "        io.prefetch();\n";
            for (int si = ps.rseg0; si < ps.rseg0 + ps.nrseg; ++si)
                emit_rev_segment(s, sc, ps, sc.rsegs[si], si == ps.rseg0 + ps.nrseg - 1);
            s << "    }\n};\n";
        }
        s << "}  // namespace\n}  // namespace dq\n";
        names.clear();
        for (int p = p0; p < p1; ++p) {
            const std::string name = "dq_jit_adj_" + std::to_string(p);
            names.push_back(name);
            s << "extern \"C\" __global__ void __launch_bounds__(" << amax << ", " << (amp == 8 && M == 4 ? 2 : 1)
              << ") " << name
              << "(const __grid_constant__ CUtensorMap mp, const __grid_constant__ CUtensorMap ml,\n"
              << "    const __grid_constant__ dq::AdjArgs a) {\n"
              << "    dq::tile_adj_body<" << R << ", " << M << ", dq::JitRev" << p << ">(mp, ml, a);\n}\n";
        }
        return s.str();
    }
    s << "#include \"dq_tile_fwd.cuh\"\n"
         "namespace dq {\nnamespace {\n";
    for (int p = p0; p < p1; ++p) {
        const TPass &ps = sc.passes[p];
        const EOp *ops = sc.ops.data() + ps.op0;
        s << "struct JitPass" << p << " {\n"
             "    template <typename R, int M, bool PD>\n"
             "    __device__ __forceinline__ static void run(cx<R> (&r)[1 << M], cx<R> *cur, const EOp *sops,\n"
             "        const ESeg *, const Mat2<R> *scoef, int, int, int, uint64_t base, int lane, int warp) {\n";
        for (int si = ps.seg0; si < ps.seg0 + ps.nseg; ++si) {
            const TSeg &sg = sc.segs[si];
            s << "    {\n        ESeg sg{}; ";
            for (int b = 0; b < M; ++b) s << "sg.B[" << b << "] = " << (int)sg.B[b] << "; ";
            s << "\n        const Layout L = make_layout(sg, M, " << sc.k << ", lane, warp);\n"
                 "        eng_load<R, M>(r, cur, L);\n";
            for (int i = sg.op0 - ps.op0; i < sg.op0 - ps.op0 + sg.nops;)
                i += emit_op(s, ops, i, ps.nops, ps.pdiag);
            s << "        eng_store<R, M>(r, cur, L);\n        __syncthreads();\n    }\n";
        }
        s << "    }\n};\n";
    }
    s << "}  // namespace\n}  // namespace dq\n";
    names.clear();
    for (int p = p0; p < p1; ++p) {
        const std::string name = "dq_jit_fwd_" + std::to_string(p);
        names.push_back(name);
        s << "extern \"C\" __global__ void __launch_bounds__(" << maxt << ", " << minb << ") " << name
          << "(const __grid_constant__ CUtensorMap tmap, dq::TileKArgs a) {\n"
          << "    dq::tile_fwd_body<" << R << ", " << M << ", " << (sc.passes[p].pdiag ? "true" : "false")
          << ", dq::JitPass" << p << ">(tmap, a);\n}\n";
    }
    return s.str();
}

bool jit_want(TileCache &tc, const std::unordered_map<uint64_t, TileTune> &tuned, const Plan &p, int amp,
              TileSchedule &sc) {
    if (tc.jit_mode == 0 || sc.jit_failed) return false;
    if (tc.jit_mode == 2) {
        auto it = tuned.find(p.key ^ (amp == 16 ? 1ull : 0ull));
        if (it == tuned.end() || it->second.jit != 1) return false;
    }
    if (!sc.jit) {
        std::string err;
        if (!jit_build(sc, amp, tc.device, &err)) {
            sc.jit_failed = true;
            tc.jit_err = err;
            return false;
        }
    }
    return true;
}

void JitModule::release() {
    for (cudaLibrary_t l : libs) cudaLibraryUnload(l);
    libs.clear();
    kernels.clear();
}

bool jit_available() {
#ifdef DQ_BOUNDS_BUILD
    return false;   // the bounds-checking build runs the (checked) interpreting kernels only
#else
    return nvrtc_api().ok;
#endif
}

bool jit_compile(const std::string &src, int cc, std::vector<char> *cubin, std::string *err) {
    NvrtcApi &api = nvrtc_api();
    if (!jit_available()) {
        if (err) *err = api.ok ? "run-time specialisation is off in the bounds-checking build" : "NVRTC is not available";
        return false;
    }
    const std::string cpath = cubin ? cache_path(src, cc) : std::string();
    if (cubin && cache_read(cpath, cubin)) return true;
    const std::string arch = "-arch=sm_" + std::to_string(cc) + "a";
    nvrtcProgram prog;
    if (api.create(&prog, src.c_str(), "dq_jit_fwd.cu", kJitHeaderCount, kJitHeaderTexts, kJitHeaderNames) !=
        NVRTC_SUCCESS) {
        if (err) *err = "nvrtcCreateProgram failed";
        return false;
    }
    const char *opts[] = {arch.c_str(), "-std=c++17", "-default-device", "-lineinfo"};
    const nvrtcResult cr = api.compile(prog, 4, opts);
    if (cr != NVRTC_SUCCESS) {
        size_t n = 0;
        api.log_size(prog, &n);
        std::string log(n + 1, '\0');
        api.log(prog, &log[0]);
        if (err) *err = "NVRTC compile failed: " + log.substr(0, 2000);
        api.destroy(&prog);
        return false;
    }
    if (cubin) {
        size_t n = 0;
        api.cubin_size(prog, &n);
        cubin->resize(n);
        api.cubin(prog, cubin->data());
        cache_write(cpath, *cubin);
    }
    api.destroy(&prog);
    return true;
}

bool jit_rows_build(RowProgram &rp, int amp, int device, std::string *err, int rpc) {
    if (rpc != 1 && rpc != 2) {
        if (err) *err = "rows per CTA must be 1 or 2";
        return false;
    }
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
    std::vector<char> cubin;
    if (!jit_compile(jit_rows_source(rp, amp, rpc), major * 10 + minor, &cubin, err)) return false;
    JitModule *m = new JitModule();
    cudaLibrary_t lib = nullptr;
    cudaError_t e = cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    cudaKernel_t k = nullptr;
    if (e == cudaSuccess) {
        m->libs.push_back(lib);
        e = cudaLibraryGetKernel(&k, lib, "dq_jit_rows");
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        m->release();
        delete m;
        if (err) *err = std::string("loading the whole-row kernel: ") + cudaGetErrorString(e);
        return false;
    }
    m->kernels.push_back(k);
    m->grid.assign(1, 0);
    m->smem_set.assign(1, 0);
    if (rp.jit[rpc - 1]) {
        rp.jit[rpc - 1]->release();
        delete rp.jit[rpc - 1];
    }
    rp.jit[rpc - 1] = m;
    return true;
}

bool jit_build(TileSchedule &sc, int amp, int device, std::string *err) {
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
    const int np = (int)sc.passes.size();
    if (np == 0) {
        if (err) *err = "empty schedule";
        return false;
    }
    // passes split into chunks compiled by concurrent NVRTC programs
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int nchunk = std::max(1, std::min({np, 8, (int)hw}));
    const int per = (np + nchunk - 1) / nchunk;
    struct Chunk {
        int p0 = 0, p1 = 0;
        std::vector<std::string> names;
        std::vector<char> cubin;
        std::string err;
        bool ok = false;
    };
    std::vector<Chunk> chunks;
    for (int p0 = 0; p0 < np; p0 += per) {
        Chunk c;
        c.p0 = p0;
        c.p1 = std::min(np, p0 + per);
        chunks.push_back(c);
    }
    std::vector<std::thread> workers;
    for (Chunk &c : chunks)
        workers.emplace_back([&sc, amp, &c, major, minor] {
            const std::string src = jit_source(sc, amp, c.names, c.p0, c.p1);
            c.ok = jit_compile(src, major * 10 + minor, &c.cubin, &c.err);
        });
    for (std::thread &t : workers) t.join();
    for (const Chunk &c : chunks)
        if (!c.ok) {
            if (err) *err = c.err;
            return false;
        }
    JitModule *m = new JitModule();
    for (const Chunk &c : chunks) {
        cudaLibrary_t lib = nullptr;
        cudaError_t e = cudaLibraryLoadData(&lib, c.cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
        if (e != cudaSuccess) {
            cudaGetLastError();
            m->release();
            delete m;
            if (err) *err = std::string("cudaLibraryLoadData: ") + cudaGetErrorString(e);
            return false;
        }
        m->libs.push_back(lib);
        for (const std::string &name : c.names) {
            cudaKernel_t k = nullptr;
            e = cudaLibraryGetKernel(&k, lib, name.c_str());
            if (e != cudaSuccess) {
                cudaGetLastError();
                m->release();
                delete m;
                if (err) *err = std::string("cudaLibraryGetKernel: ") + cudaGetErrorString(e);
                return false;
            }
            m->kernels.push_back(k);
        }
    }
    m->grid.assign(m->kernels.size(), 0);
    m->smem_set.assign(m->kernels.size(), 0);
    if (sc.jit) {
        sc.jit->release();
        delete sc.jit;
    }
    sc.jit = m;
    return true;
}

}  // namespace dq
