// persist.cuh -- host-side file formats of the context: the checkpoint (one
// line of JSON header, then raw little-endian fp32 arrays) and the autotune
// cache (JSON lines).  Only the flat objects this library writes are read:
// numbers, strings and arrays of numbers.
#pragma once
#include <cstddef>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

namespace drc {

// 64-bit FNV-1a of a byte range (continue from h).
uint64_t fnv1a64(const void *p, size_t n, uint64_t h = 1469598103934665603ull);

// A flat JSON object: each key's value as its source text.
struct FlatJson {
  std::map<std::string, std::string> raw;
  bool num(const std::string &k, double *v) const;
  bool str(const std::string &k, std::string *v) const;
  bool nums(const std::string &k, std::vector<double> *v) const;
};
// Parse one object (one line); false on anything outside the flat form.
bool parse_flat_json(const std::string &text, FlatJson *out);
// JSON string literal of s (quotes, backslashes and control characters escaped).
std::string json_quote(const std::string &s);

// Write header + "\n" + the blobs to path through a temporary file renamed
// over it (readers never see a partial file).  false with errno set on failure.
bool write_file_atomic(const std::string &path, const std::string &header,
                       const std::vector<std::pair<const void *, size_t>> &blobs);
bool read_file(const std::string &path, std::string *data);
// Append one line (with its newline) in a single write.
bool append_line(const std::string &path, const std::string &line);

}  // namespace drc
