// A scoped NVTX range on the calling host thread (the enqueue span of a
// generation, a batched step or a serving step), carrying an integer payload
// (the generation index, the count).  NVTX v3 is header-only; without a tool
// attached each call is a check of a function pointer.
#pragma once
#include <nvtx3/nvToolsExt.h>

#include <cstdint>

namespace rvea {

class NvtxRange {
 public:
  NvtxRange(const char *name, int64_t payload) {
    nvtxEventAttributes_t a = {};
    a.version = NVTX_VERSION;
    a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
    a.messageType = NVTX_MESSAGE_TYPE_ASCII;
    a.message.ascii = name;
    a.payloadType = NVTX_PAYLOAD_TYPE_INT64;
    a.payload.llValue = payload;
    nvtxRangePushEx(&a);
  }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace rvea
