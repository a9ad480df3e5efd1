// Batched stepping of many independent simulations (the paper's parameter-scan workload:
// scans over stencil order, resolution and propagation length, section "Accurate
// modeling of plasma accelerators in finite order PSATD").
//
// The cycles of all simulations are captured once into a single CUDA graph: each
// simulation keeps its own stream, forked from and joined back to the caller's origin
// stream, so simulations of uneven size run concurrently and one graph launch advances
// all of them with no per-kernel host work.  The particle double buffers flip once per
// cycle, so a graph holds an even number of cycles and the buffers return to their
// starting parity after every launch.
#include <new>
#include <vector>

#include "pic_internal.cuh"

namespace pic {
pic_status step_cycle(Sim* s);   // pic_api.cu: one full cycle on s->stream
}

using namespace pic;

struct pic_batch {
  std::vector<Sim*> sims;
  cudaStream_t origin = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int32_t cycles = 0;
  int64_t kernels_per_launch = 0;
  std::vector<cudaEvent_t> events;
};

static void batch_free(pic_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaEvent_t e : b->events) cudaEventDestroy(e);
  delete b;
}

extern "C" pic_status pic_batch_create(pic_sim* const* sims, int32_t n_sims, int32_t cycles_per_launch,
                                       void* origin_stream, pic_batch** out) {
  if (!out) { set_error("out is NULL"); return PIC_ERR_ARG; }
  *out = nullptr;
  if (!sims || n_sims < 1) { set_error("need at least one simulation"); return PIC_ERR_ARG; }
  if (cycles_per_launch < 2 || (cycles_per_launch & 1)) {
    set_error("cycles_per_launch=%d must be even and >= 2", cycles_per_launch);
    return PIC_ERR_ARG;
  }
  if (!origin_stream) { set_error("the origin stream must be a created (non-default) stream"); return PIC_ERR_ARG; }
  pic_batch* b = new (std::nothrow) pic_batch;
  if (!b) { set_error("host allocation failed"); return PIC_ERR_OOM; }
  b->origin = reinterpret_cast<cudaStream_t>(origin_stream);
  b->cycles = cycles_per_launch;
  for (int i = 0; i < n_sims; ++i) {
    Sim* s = reinterpret_cast<Sim*>(sims[i]);
    if (!s || !s->fields_ready || !s->stream) {
      set_error("simulation %d is NULL, not initialised, or on the default stream", i);
      batch_free(b);
      return PIC_ERR_ARG;
    }
    if (s->win.on) {   // a captured graph would replay one window position forever
      set_error("simulation %d has a moving window; batches take fixed windows only", i);
      batch_free(b);
      return PIC_ERR_ARG;
    }
    b->sims.push_back(s);
  }
  b->events.resize(n_sims + 1);
  for (auto& e : b->events) {
    cudaError_t ce = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    if (ce != cudaSuccess) { e = nullptr; batch_free(b); return cuda_status(ce, "cudaEventCreate"); }
  }
  // finish any pending work first: capture requires idle, non-legacy streams
  for (Sim* s : b->sims) {
    cudaError_t ce = cudaStreamSynchronize(s->stream);
    if (ce != cudaSuccess) { batch_free(b); return cuda_status(ce, "cudaStreamSynchronize"); }
  }
  int64_t before = 0;
  for (Sim* s : b->sims) before += s->launches;
  cudaError_t ce = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal);
  if (ce != cudaSuccess) { batch_free(b); return cuda_status(ce, "cudaStreamBeginCapture"); }
  pic_status st = PIC_OK;
  if ((ce = cudaEventRecord(b->events[0], b->origin)) != cudaSuccess) st = cuda_status(ce, "cudaEventRecord");
  for (size_t i = 0; st == PIC_OK && i < b->sims.size(); ++i)
    if ((ce = cudaStreamWaitEvent(b->sims[i]->stream, b->events[0], 0)) != cudaSuccess)
      st = cuda_status(ce, "cudaStreamWaitEvent");
  for (int k = 0; st == PIC_OK && k < b->cycles; ++k)
    for (size_t i = 0; st == PIC_OK && i < b->sims.size(); ++i) st = step_cycle(b->sims[i]);
  for (size_t i = 0; st == PIC_OK && i < b->sims.size(); ++i) {
    if ((ce = cudaEventRecord(b->events[i + 1], b->sims[i]->stream)) != cudaSuccess)
      st = cuda_status(ce, "cudaEventRecord");
    else if ((ce = cudaStreamWaitEvent(b->origin, b->events[i + 1], 0)) != cudaSuccess)
      st = cuda_status(ce, "cudaStreamWaitEvent");
  }
  cudaGraph_t g = nullptr;
  ce = cudaStreamEndCapture(b->origin, &g);
  b->graph = g;
  if (st != PIC_OK) { batch_free(b); return st; }
  if (ce != cudaSuccess) { batch_free(b); return cuda_status(ce, "cudaStreamEndCapture"); }
  if ((ce = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess) {
    b->exec = nullptr;
    batch_free(b);
    return cuda_status(ce, "cudaGraphInstantiate");
  }
  int64_t after = 0;
  for (Sim* s : b->sims) after += s->launches;
  b->kernels_per_launch = after - before;
  // the capture ran the host side of every cycle: the particle buffers flipped an even
  // number of times, so each handle's current buffer is unchanged
  *out = b;
  return PIC_OK;
}

extern "C" pic_status pic_batch_launch(pic_batch* b, int32_t n_launches) {
  if (!b) { set_error("batch is NULL"); return PIC_ERR_ARG; }
  if (n_launches < 0) { set_error("n_launches=%d < 0", n_launches); return PIC_ERR_ARG; }
  for (int32_t i = 0; i < n_launches; ++i) {
    cudaError_t ce = cudaGraphLaunch(b->exec, b->origin);
    if (ce != cudaSuccess) return cuda_status(ce, "cudaGraphLaunch");
  }
  return PIC_OK;
}

extern "C" pic_status pic_batch_info(pic_batch* b, int32_t* cycles_per_launch, int64_t* kernels_per_launch) {
  if (!b) { set_error("batch is NULL"); return PIC_ERR_ARG; }
  if (cycles_per_launch) *cycles_per_launch = b->cycles;
  if (kernels_per_launch) *kernels_per_launch = b->kernels_per_launch;
  return PIC_OK;
}

extern "C" pic_status pic_batch_destroy(pic_batch* b) {
  batch_free(b);
  return PIC_OK;
}
