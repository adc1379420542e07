// Autotuner: picks, per plan and block size, the compiled tier's threads
// per CTA (tile = 4 bytes x threads per strip) and the register budget that
// bounds the XorRePair temporaries (Sec. 4.4 compression against Sec. 6
// pebble/register pressure), by timing each candidate on scratch stripes.
// Every candidate's parity is compared with the first one's; the fastest
// program replaces the plan's encoder and later decode programs inherit the
// budget and launch shape.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "gf.h"
#include "internal.h"

using xorec::Program;

namespace xorec {

int minb_for(int threads, int reg_budget) {
  const int per_sm_regs = 65536;
  int minb = per_sm_regs / (threads * reg_budget);
  if (minb < 1) minb = 1;
  if (minb * threads > 1024) minb = 1024 / threads;
  return minb;
}

}  // namespace xorec

namespace {

struct Candidate {
  int threads, reg_budget;
};


// Make `prog` the plan's encoder and (threads, reg_budget) the launch shape
// of the plan's compiled programs and batch modules built from now on.
void install(ec_plan* plan, std::unique_ptr<Program> prog, int threads, int reg_budget) {
  std::lock_guard<std::mutex> lk(plan->mu);
  // the old encoder may still be referenced by existing batches: retire it
  plan->retired.push_back(std::move(plan->enc));
  plan->enc = std::move(prog);
  plan->opts.reg_budget = reg_budget;
  plan->opts.max_temps = -2;
  plan->tuned_threads = threads;
  plan->tuned_minb = xorec::minb_for(threads, reg_budget);
}

}  // namespace

extern "C" ec_status ec_plan_set_launch(ec_plan* plan, int threads, int reg_budget) {
  if (!plan) return fail(EC_EINVAL, "NULL plan");
  if (threads < 32 || threads > 1024 || threads % 32 != 0)
    return fail(EC_EINVAL, "threads must be a multiple of 32 in [32, 1024]");
  if (reg_budget < 32 || reg_budget > 255) return fail(EC_EINVAL, "reg_budget must be in [32, 255]");
  xorec::PlanOptions o = plan->opts;
  o.reg_budget = reg_budget;
  o.max_temps = -2;
  auto prog = std::make_unique<Program>();
  std::string err;
  if (!xorec::build_program(plan->m, plan->k, plan->P.data(), o, prog.get(), &err))
    return fail(EC_EINVAL, err);
  prog->threads = threads;
  prog->minb = xorec::minb_for(threads, reg_budget);
  install(plan, std::move(prog), threads, reg_budget);
  return EC_OK;
}

extern "C" ec_status ec_plan_autotune(ec_plan* plan, size_t block_bytes, int n_stripes,
                                      void* stream, ec_tune_result* out) {
  xorec::TraceRange trace_("xorec autotune");
  if (!plan) return fail(EC_EINVAL, "NULL plan");
  if (block_bytes == 0 || block_bytes % 128 != 0)
    return fail(EC_EINVAL, "block_bytes must be a positive multiple of 128");
  if (n_stripes < 1) return fail(EC_EINVAL, "need at least one stripe");
  if (!xorec::jit_available()) return fail(EC_ENOTSUP, "no run-time compiler available");
  xorec::DeviceInfo di;
  if (!xorec::device_info(&di)) return EC_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int k = plan->k, m = plan->m;
  const size_t din = static_cast<size_t>(k) * block_bytes, dout = static_cast<size_t>(m) * block_bytes;
  uint8_t *d_in = nullptr, *d_out = nullptr;
  if (xorec::dev_malloc(&d_in, n_stripes * din) != cudaSuccess ||
      xorec::dev_malloc(&d_out, n_stripes * dout) != cudaSuccess) {
    cudaGetLastError();
    if (d_in) cudaFree(d_in);
    return fail(EC_ENOMEM, "scratch allocation for tuning failed");
  }
  if (!xorec::launch_synth_fill(d_in, n_stripes * din, 0x7475e5ull, 0, st)) {
    cudaFree(d_in);
    cudaFree(d_out);
    return EC_ECUDA;
  }
  std::vector<Candidate> cands = {{128, 128}, {128, 112}, {128, 96}, {128, 160}, {256, 128},
                                  {256, 112}};
  // wide codes: also the narrower tiles that keep two CTAs per SM
  const int wide_threads = xorec::tile_threads_for_inputs(8 * k, 128);
  if (wide_threads < 128)
    for (int b : {128, 160, 112}) cands.push_back(Candidate{wide_threads, b});
  std::vector<uint8_t> ref, got(n_stripes * dout);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  xk::IoDesc io;
  std::memset(&io, 0, sizeof(io));
  io.in_base = d_in;
  io.in_sstride = static_cast<long long>(din);
  io.in_bstride = static_cast<long long>(block_bytes);
  io.out_base = d_out;
  io.out_sstride = static_cast<long long>(dout);
  io.out_bstride = static_cast<long long>(block_bytes);
  io.n_inblk = k;
  io.n_outblk = m;
  io.S = static_cast<long long>(block_bytes / 8);
  io.n_stripes = n_stripes;
  float best_ms = 1e30f;
  int best = -1, tried = 0;
  std::unique_ptr<Program> best_prog;
  ec_status rc = EC_OK;
  for (int c = 0; c < static_cast<int>(cands.size()); ++c) {
    xorec::PlanOptions o = plan->opts;
    o.reg_budget = cands[c].reg_budget;
    if (o.max_temps != -2) o.max_temps = -2;
    auto prog = std::make_unique<Program>();
    std::string err;
    if (!xorec::build_program(m, k, plan->P.data(), o, prog.get(), &err)) {
      rc = fail(EC_EINVAL, err);
      break;
    }
    prog->threads = cands[c].threads;
    prog->minb = xorec::minb_for(cands[c].threads, cands[c].reg_budget);
    if (!xorec::single_launch_fits(prog.get(), prog->threads, di.smem_optin)) continue;
    if (!xorec::launch_program(prog.get(), io, EC_EXEC_COMPILED, st)) {   // compiles
      xorec::jit_release(prog.get());
      continue;
    }
    for (int w = 0; w < 2; ++w) xorec::launch_program(prog.get(), io, EC_EXEC_COMPILED, st);
    cudaEventRecord(e0, st);
    const int reps = 5;
    for (int r = 0; r < reps; ++r) xorec::launch_program(prog.get(), io, EC_EXEC_COMPILED, st);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess ||
        cudaMemcpy(got.data(), d_out, got.size(), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      xorec::jit_release(prog.get());
      rc = fail(EC_ECUDA, "tuning run failed");
      break;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= reps;
    ++tried;
    if (ref.empty()) {
      ref = got;
    } else if (ref != got) {
      xorec::jit_release(prog.get());
      rc = fail(EC_ECUDA, "tuning candidates disagree");
      break;
    }
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
      if (best_prog) xorec::jit_release(best_prog.get());
      best_prog = std::move(prog);
    } else {
      xorec::jit_release(prog.get());
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d_in);
  cudaFree(d_out);
  if (rc != EC_OK) {
    if (best_prog) xorec::jit_release(best_prog.get());
    return rc;
  }
  if (best < 0) return fail(EC_ENOTSUP, "no candidate fits the compiled tier");
  // install: encoder program, budget and launch shape for later decoders
  install(plan, std::move(best_prog), cands[best].threads, cands[best].reg_budget);
  if (out) {
    out->threads = cands[best].threads;
    out->reg_budget = cands[best].reg_budget;
    out->min_ctas_per_sm = xorec::minb_for(cands[best].threads, cands[best].reg_budget);
    out->candidates = tried;
    out->ms = best_ms;
    out->gbps_in = static_cast<double>(n_stripes) * din / (best_ms / 1e3) / 1e9;
  }
  return EC_OK;
}
