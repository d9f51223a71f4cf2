// Round loops as CUDA graphs: one conditional while node whose body is
// captured from the launches a caller makes on a capture stream; the body's
// last kernel sets the loop condition with cudaGraphSetConditional.  A
// context keeps one such graph per loop (ADG's rounds, the segmented batch
// path's rounds), keyed by the bytes of everything the captured launches bake
// in (buffer addresses, grid shapes): it is built on the second call in a row
// with the same key -- building costs more than a few host-driven rounds, so
// calls whose buffers keep changing stay on the host loop -- and launched as
// is while the key stays the same.
#include <cstring>
#include <new>

#include "gc_internal.cuh"

namespace gc {

namespace {
void release(LoopGraph* lg) {
  if (lg->exec) cudaGraphExecDestroy(lg->exec);
  if (lg->graph) cudaGraphDestroy(lg->graph);
  lg->exec = nullptr;
  lg->graph = nullptr;
}
}  // namespace

cudaError_t loop_graph(LoopGraph** slot, const void* key, size_t key_bytes,
                       const std::function<void(cudaStream_t, cudaGraphConditionalHandle)>& capture,
                       cudaGraphExec_t* exec) {
  const unsigned char* k = static_cast<const unsigned char*>(key);
  LoopGraph* lg = *slot;
  auto same = [&](const std::vector<unsigned char>& v) {
    return v.size() == key_bytes && memcmp(v.data(), k, key_bytes) == 0;
  };
  if (lg && lg->exec && same(lg->key)) {
    *exec = lg->exec;
    return cudaSuccess;
  }
  if (!lg) {
    lg = new (std::nothrow) LoopGraph();
    if (!lg) return cudaErrorMemoryAllocation;
    *slot = lg;
  }
  if (!same(lg->seen)) {  // first call with this key: the caller's host loop
    lg->seen.assign(k, k + key_bytes);
    return cudaErrorNotReady;
  }
  release(lg);
  cudaGraph_t graph = nullptr;
  cudaStream_t cs = nullptr;
  cudaGraphExec_t ex = nullptr;
  cudaError_t e = cudaGraphCreate(&graph, 0);
  do {
    if (e != cudaSuccess) break;
    cudaGraphConditionalHandle loop;
    if ((e = cudaGraphConditionalHandleCreate(&loop, graph, 1, cudaGraphCondAssignDefault)) != cudaSuccess) break;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = loop;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp)) != cudaSuccess) break;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) break;
    if ((e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
      break;
    capture(cs, loop);
    cudaGraph_t captured = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(cs, &captured);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = ec) != cudaSuccess) break;
    e = cudaGraphInstantiate(&ex, graph, 0);
  } while (false);
  if (cs) cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (ex) cudaGraphExecDestroy(ex);
    if (graph) cudaGraphDestroy(graph);
    return e;
  }
  lg->key.assign(k, k + key_bytes);
  lg->graph = graph;
  lg->exec = ex;
  *exec = ex;
  return cudaSuccess;
}

void loop_graph_free(LoopGraph** slot) {
  if (!*slot) return;
  release(*slot);
  delete *slot;
  *slot = nullptr;
}

}  // namespace gc
