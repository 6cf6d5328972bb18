// persist.cu -- host-side file helpers of the checkpoint and the autotune
// cache (see persist.cuh).
#include "persist.cuh"

#include <fcntl.h>
#include <unistd.h>

#include <cerrno>
#include <cstdio>
#include <cstdlib>
#include <cstring>

namespace drc {

uint64_t fnv1a64(const void *p, size_t n, uint64_t h) {
  const unsigned char *b = static_cast<const unsigned char *>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

namespace {

void skip_ws(const std::string &t, size_t &i) {
  while (i < t.size() && (t[i] == ' ' || t[i] == '\t' || t[i] == '\n' || t[i] == '\r')) ++i;
}

// A string literal starting at t[i] == '"': its decoded text; i moves past it.
bool read_string(const std::string &t, size_t &i, std::string *out) {
  if (i >= t.size() || t[i] != '"') return false;
  std::string s;
  for (++i; i < t.size(); ++i) {
    const char ch = t[i];
    if (ch == '"') {
      ++i;
      if (out) *out = s;
      return true;
    }
    if (ch == '\\') {
      if (++i >= t.size()) return false;
      const char e = t[i];
      if (e == 'n') s += '\n';
      else if (e == 't') s += '\t';
      else if (e == 'r') s += '\r';
      else if (e == '"' || e == '\\' || e == '/') s += e;
      else return false;  // \uXXXX and others: not written by this library
    } else {
      s += ch;
    }
  }
  return false;
}

}  // namespace

bool parse_flat_json(const std::string &t, FlatJson *out) {
  size_t i = 0;
  skip_ws(t, i);
  if (i >= t.size() || t[i] != '{') return false;
  ++i;
  out->raw.clear();
  skip_ws(t, i);
  if (i < t.size() && t[i] == '}') return true;
  while (i < t.size()) {
    skip_ws(t, i);
    std::string key;
    if (!read_string(t, i, &key)) return false;
    skip_ws(t, i);
    if (i >= t.size() || t[i] != ':') return false;
    ++i;
    skip_ws(t, i);
    const size_t v0 = i;
    if (i < t.size() && t[i] == '"') {
      if (!read_string(t, i, nullptr)) return false;
    } else if (i < t.size() && t[i] == '[') {
      while (i < t.size() && t[i] != ']') {
        if (t[i] == '[' && i != v0) return false;  // arrays of arrays are not part of the form
        if (t[i] == '"' || t[i] == '{') return false;
        ++i;
      }
      if (i >= t.size()) return false;
      ++i;
    } else {
      while (i < t.size() && t[i] != ',' && t[i] != '}') {
        if (t[i] == '{' || t[i] == '[' || t[i] == '"') return false;
        ++i;
      }
    }
    std::string val = t.substr(v0, i - v0);
    while (!val.empty() && (val.back() == ' ' || val.back() == '\t')) val.pop_back();
    out->raw[key] = val;
    skip_ws(t, i);
    if (i < t.size() && t[i] == ',') {
      ++i;
      continue;
    }
    if (i < t.size() && t[i] == '}') return true;
    return false;
  }
  return false;
}

bool FlatJson::num(const std::string &k, double *v) const {
  auto it = raw.find(k);
  if (it == raw.end() || it->second.empty()) return false;
  char *end = nullptr;
  const double d = strtod(it->second.c_str(), &end);
  if (!end || *end) {
    if (it->second == "true") *v = 1;
    else if (it->second == "false") *v = 0;
    else return false;
    return true;
  }
  *v = d;
  return true;
}

bool FlatJson::str(const std::string &k, std::string *v) const {
  auto it = raw.find(k);
  if (it == raw.end()) return false;
  size_t i = 0;
  return read_string(it->second, i, v) && i == it->second.size();
}

bool FlatJson::nums(const std::string &k, std::vector<double> *v) const {
  auto it = raw.find(k);
  if (it == raw.end()) return false;
  const std::string &t = it->second;
  if (t.size() < 2 || t.front() != '[' || t.back() != ']') return false;
  v->clear();
  size_t i = 1;
  while (i < t.size() - 1) {
    skip_ws(t, i);
    if (i >= t.size() - 1) break;
    char *end = nullptr;
    const double d = strtod(t.c_str() + i, &end);
    if (end == t.c_str() + i) return false;
    v->push_back(d);
    i = (size_t)(end - t.c_str());
    skip_ws(t, i);
    if (i < t.size() - 1) {
      if (t[i] != ',') return false;
      ++i;
    }
  }
  return true;
}

std::string json_quote(const std::string &s) {
  std::string o = "\"";
  for (char ch : s) {
    if (ch == '"' || ch == '\\') {
      o += '\\';
      o += ch;
    } else if (ch == '\n') {
      o += "\\n";
    } else if (ch == '\t') {
      o += "\\t";
    } else if (ch == '\r') {
      o += "\\r";
    } else if ((unsigned char)ch < 0x20) {
      o += ' ';
    } else {
      o += ch;
    }
  }
  return o + "\"";
}

bool write_file_atomic(const std::string &path, const std::string &header,
                       const std::vector<std::pair<const void *, size_t>> &blobs) {
  const std::string tmp = path + ".tmp." + std::to_string((long)getpid());
  FILE *f = fopen(tmp.c_str(), "wb");
  if (!f) return false;
  bool ok = fwrite(header.data(), 1, header.size(), f) == header.size() && fputc('\n', f) != EOF;
  for (const auto &b : blobs)
    if (ok && b.second) ok = fwrite(b.first, 1, b.second, f) == b.second;
  ok = fflush(f) == 0 && ok;
  ok = fclose(f) == 0 && ok;
  if (ok) ok = rename(tmp.c_str(), path.c_str()) == 0;
  if (!ok) {
    const int keep = errno;
    remove(tmp.c_str());
    errno = keep;
  }
  return ok;
}

bool read_file(const std::string &path, std::string *data) {
  FILE *f = fopen(path.c_str(), "rb");
  if (!f) return false;
  data->clear();
  char buf[1 << 16];
  size_t n;
  while ((n = fread(buf, 1, sizeof buf, f)) > 0) data->append(buf, n);
  const bool ok = !ferror(f);
  fclose(f);
  return ok;
}

bool append_line(const std::string &path, const std::string &line) {
  const int fd = open(path.c_str(), O_WRONLY | O_CREAT | O_APPEND, 0644);
  if (fd < 0) return false;
  const std::string l = line + "\n";
  const ssize_t w = write(fd, l.data(), l.size());
  const bool ok = w == (ssize_t)l.size();
  const int keep = errno;
  close(fd);
  errno = keep;
  return ok;
}

}  // namespace drc
