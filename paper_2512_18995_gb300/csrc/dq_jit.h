// Run-time specialised tile passes and whole-row kernels (internal interface).
#pragma once

#include <cuda_runtime.h>

#include <stdint.h>

#include <string>
#include <unordered_map>
#include <vector>

namespace dq {

struct TileSchedule;
struct RowProgram;
struct TileCache;
struct TileTune;
struct Plan;

// The compiled passes of one schedule (one library, one kernel per pass).
struct JitModule {
    std::vector<cudaLibrary_t> libs;   // one per chunk of passes
    std::vector<cudaKernel_t> kernels;
    std::vector<int> grid;        // launch grid per pass for the last state buffer (0: not computed)
    std::vector<size_t> smem_set; // dynamic shared memory the kernel was opened up to
    void release();
};

bool jit_available();
// Source of the schedule's specialised passes [p0, p1) (all: p1 < 0); names
// receives the kernels'.
std::string jit_source(const TileSchedule &sc, int amp, std::vector<std::string> &names, int p0 = 0, int p1 = -1);
// Compile a source of jit_source for compute capability cc (e.g. 103 for
// sm_103a); cubin may be null (compile check only).
bool jit_compile(const std::string &src, int cc, std::vector<char> *cubin, std::string *err);
// Whether a schedule's passes run as specialised kernels (DQ_OPT_JIT on, or
// automatic with the autotuner having measured them faster for the plan);
// compiles them on first use.  A failed compile keeps the interpreter for
// that schedule (the reason in tc.jit_err).  Reverse schedules follow the
// circuit's forward decision.
bool jit_want(TileCache &tc, const std::unordered_map<uint64_t, TileTune> &tuned, const Plan &p, int amp,
              TileSchedule &sc);
// Compile and load every pass of sc for `device` (sc.jit); false with *err on failure.
bool jit_build(TileSchedule &sc, int amp, int device, std::string *err);
// Source of the whole-row kernel with the program's ops compiled in (kernel
// dq_jit_rows, taking RowArgs like the interpreting kernel; rpc rows per CTA).
std::string jit_rows_source(const RowProgram &rp, int amp, int rpc = 1);
// Compile and load it for `device` and rpc rows per CTA (rp.jit[rpc - 1], one
// kernel); false with *err on failure.
bool jit_rows_build(RowProgram &rp, int amp, int device, std::string *err, int rpc = 1);

}  // namespace dq
