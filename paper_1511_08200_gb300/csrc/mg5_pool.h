// mg5_pool.h -- captured solves as reusable entries (library-internal).
//
// An entry is one solve from zero (MG5_MIXED, or MG5_FP64 without the
// full-multigrid start) of one grid size and parameter set captured as a
// CUDA graph, with its own hierarchy, scalars, staging buffers and a pinned
// host block the solve's control state is copied into.  A context keeps its
// entries in a list; an entry is busy from checkout until its result has been
// read, so one entry never runs twice at once.  The functions that touch a
// context's list are not thread-safe: a context used from several threads (the
// server's pool) guards them with its own lock.  graph_build captures on
// private streams and allocates: the caller keeps other threads from freeing
// device memory or synchronising the device meanwhile, since either may end a
// capture in progress.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <string>

#include "mg5.h"

struct GraphEntry;

namespace mg5 {

// Device bytes one entry of that precision holds.
size_t graph_bytes(int N, int precision, bool grad);
// Whether a solve of (N, p) can be captured: MG5_MIXED always; MG5_FP64 with two grids or
// more and nu1 + nu2 even (the loop body must return every grid to its buffer).
bool graph_capturable(int N, const mg5_params *p);
// An idle entry of ctx for (N, p, grad), marked busy; nullptr if there is none.
GraphEntry *graph_checkout(mg5_ctx *ctx, int N, const mg5_params *p, bool grad);
// Build (allocate + capture + instantiate) a new MG5_MIXED entry on `device`, not yet in any list.
int graph_build(int device, int N, const mg5_params *p, bool grad, GraphEntry **out,
                std::string *err);
// Build a new entry of p's precision on ctx's device (MG5_FP64 reads ctx's profiler switch and
// writes its error text: the caller serialises builds on one ctx), not yet in any list.
int graph_build_in(mg5_ctx *ctx, int N, const mg5_params *p, bool grad, GraphEntry **out,
                   std::string *err);
// Add a built entry to ctx's list (busy) and count its bytes in ctx.
void graph_insert(mg5_ctx *ctx, GraphEntry *g);
// Remove ctx's least recently used idle entry from its list (bytes uncounted); nullptr if none.
GraphEntry *graph_take_idle(mg5_ctx *ctx);
// Free an entry that is in no list.
void graph_free(GraphEntry *g);
// Enqueue on st: copy delta in, launch, copy phi (and grad) out, copy the control state to host.
int graph_enqueue(GraphEntry *g, const double *delta, double *phi, double *grad, cudaStream_t st,
                  std::string *err);
// After st has synchronised: the solve's status and info; the entry becomes idle.
int graph_finish(GraphEntry *g, mg5_info *info);
// Return an entry whose solve failed, idle, without reading its result.
void graph_checkin(GraphEntry *g);
// Entries ctx holds for (N, p, grad), busy or idle.
int graph_count(mg5_ctx *ctx, int N, const mg5_params *p, bool grad);
// Bytes ctx holds in entries.
size_t graph_held(mg5_ctx *ctx);

}  // namespace mg5
