// Host-only harness for hd_exact.cuh (no GPU): reads little-endian doubles
// from argv[1], sums them into one Exact192 in file order and, separately,
// in chunks of argv[2] values merged last chunk first, and prints the two
// rounded sums as 64-bit patterns in hex.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "hd_exact.cuh"

int main(int argc, char** argv) {
    if (argc < 3) return 2;
    FILE* f = std::fopen(argv[1], "rb");
    if (!f) return 2;
    std::vector<double> v;
    double x;
    while (std::fread(&x, sizeof x, 1, f) == 1) v.push_back(x);
    std::fclose(f);
    const size_t chunk = size_t(std::strtoull(argv[2], nullptr, 10));
    hd::Exact192 a = hd::exact_zero();
    for (double t : v) hd::exact_add(a, t);
    std::vector<hd::Exact192> parts;
    for (size_t i = 0; i < v.size(); i += chunk) {
        hd::Exact192 p = hd::exact_zero();
        for (size_t j = i; j < v.size() && j < i + chunk; ++j) hd::exact_add(p, v[j]);
        parts.push_back(p);
    }
    hd::Exact192 b = hd::exact_zero();
    for (size_t i = parts.size(); i-- > 0;) hd::exact_merge(b, parts[i]);
    std::printf("%016llx %016llx\n", hd::exact_bits(hd::exact_round(a)), hd::exact_bits(hd::exact_round(b)));
    return 0;
}
