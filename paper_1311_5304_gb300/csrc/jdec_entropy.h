// jdec_entropy.h -- internal interface of the host entropy decoder used by
// the pipelined JPEG decoder: a parsed stream whose MCU rows can be decoded
// in order (one resumable decoder) or in independent chunks that start at
// restart intervals (several host threads).
#pragma once

#include <cstddef>
#include <cstdint>

#include "../../include/jdec.h"

namespace jdec {

struct JpegScan;

jdec_status scan_open(const uint8_t *data, size_t size, JpegScan **out, jdec_jpeg_info *info);
void scan_close(JpegScan *J);
int scan_row_step(const JpegScan *J);
jdec_status scan_prepare_independent(JpegScan *J);
jdec_status scan_decode_rows(JpegScan *J, int16_t *const planes[3], int r0, int r1, bool independent);

}  // namespace jdec
