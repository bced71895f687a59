"""Random-access ceiling of the GPU's memory: scattered 4-, 8- and 16-byte
reads and 8-byte writes over an array far larger than L2.

The bottom-up and top-down steps of BFS touch memory mostly as scattered
accesses of 4 to 16 bytes (a vertex's (first, degree) pair, a (level,
parent) entry, a frontier word). DRAM moves a whole 32-byte sector for each,
and scattered sectors stream more slowly than a copy. This tool measures how
many such accesses per second the memory system sustains
(`dobfs_debug_random_access`: positions from a hash, eight accesses in
flight per thread, every SM busy), next to the streaming copy bandwidth
that the roofline fractions use. PyTorch's own 8-byte gather
(`index_select`, which also reads an index array) is timed beside it as a
reference.

    python -m paper_1503_04359_b300.gather_peak [--gb 4] [--m 268435456] [--json]
"""
import argparse
import json
import sys


def measure(gb: int = 4, m: int = 1 << 28, torch_reference: bool = True) -> dict:
    from paper_1503_04359_b300 import dobfs

    dobfs.load()
    array_bytes = int(gb) << 30
    out = {"array_gb": gb, "accesses": m, "cases": {}}
    for name, width, write in (("read4", 4, False), ("read8", 8, False), ("read16", 16, False),
                               ("write8", 8, True)):
        ms, made = dobfs.dobfs_debug_random_access(array_bytes, m, width, write)
        rate = made / (ms * 1e-3)
        out["cases"][name] = {"ms": ms, "accesses": made, "accesses_per_s": rate,
                              "useful_gbs": rate * width / 1e9, "sector_gbs": rate * 32 / 1e9}
    if torch_reference:
        import torch

        gen = torch.Generator(device="cuda")
        gen.manual_seed(1)
        arr = torch.zeros(array_bytes // 8, dtype=torch.int64, device="cuda")
        k = min(m, 1 << 26)
        idx = torch.randint(0, arr.numel(), (k,), generator=gen, device="cuda")
        arr.index_select(0, idx)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        arr.index_select(0, idx)
        e.record()
        torch.cuda.synchronize()
        ms = s.elapsed_time(e)
        rate = k / (ms * 1e-3)
        out["cases"]["torch_index_select8"] = {"ms": ms, "accesses": k, "accesses_per_s": rate,
                                               "useful_gbs": rate * 8 / 1e9, "sector_gbs": rate * 32 / 1e9}
        del arr, idx
        torch.cuda.empty_cache()
    return out


def main() -> int:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gb", type=int, default=4, help="array size in GB, a power of two (far above the 126 MB L2)")
    ap.add_argument("--m", type=int, default=1 << 28, help="accesses per launch")
    ap.add_argument("--no-torch", action="store_true", help="skip PyTorch's gather")
    ap.add_argument("--json", action="store_true")
    args = ap.parse_args()
    r = measure(args.gb, args.m, not args.no_torch)
    if args.json:
        print(json.dumps(r))
        return 0
    print("array %d GB" % r["array_gb"])
    for name, c in r["cases"].items():
        print("%-20s %9.3f ms  %6.1f G accesses/s  useful %7.1f GB/s  sectors %7.1f GB/s"
              % (name, c["ms"], c["accesses_per_s"] / 1e9, c["useful_gbs"], c["sector_gbs"]))
    return 0


if __name__ == "__main__":
    sys.exit(main())
