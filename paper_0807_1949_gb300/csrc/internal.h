// Internal declarations shared by the host sources of libvtm (not part of the C ABI).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/vtm.h"

namespace vtm {

// Error carrying a vtm_status code; caught at the C ABI boundary.
struct Error {
  int code;
  std::string msg;
};

[[noreturn]] void fail(int code, const std::string& msg);
void set_last_error(const std::string& msg);
// Puts the allocation-free residual's scratch array on the current device (noalloc.cu).
void noalloc_prepare_current_device();

}  // namespace vtm

// The split electric graph G̃_e (§4): copies numbered piece by piece, local matrices Ã_j in
// local CSR, source shares and lines.  Plus a copy of A for the FP64 residual.
struct vtm_partition {
  int64_t n = 0;
  int32_t npieces = 0;
  std::vector<int64_t> a_rowptr;
  std::vector<int32_t> a_col;
  std::vector<double> a_val;

  std::vector<int64_t> piece_ptr;    // npieces+1
  std::vector<int64_t> copy_vertex;  // C
  std::vector<double> copy_share;    // C
  std::vector<int64_t> l_rowptr;     // C+1
  std::vector<int32_t> l_col;        // local column within the piece
  std::vector<double> l_val;
  std::vector<int64_t> line_a, line_b;  // copy ids of the two ends of each line
  int64_t nboundary = 0;
};
