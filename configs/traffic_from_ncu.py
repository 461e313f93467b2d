"""Writes configs/traffic.json, the DRAM traffic of the benchmark's dominant kernel, from
an ncu capture of that kernel (CSV of dram__bytes_read.sum, dram__bytes_write.sum).

The ratio of measured DRAM bytes to the kernel's algorithmic bytes (each link, input and
output moved once) is stored together with a hash of the stencil sources; bench.py
reports traffic = ratio x algorithmic bytes per launch while the sources still match,
and null otherwise.

usage: python configs/traffic_from_ncu.py CSV --name dslash_cg_f32_k16 --sites V --k K --links 12|18
       --variant N [--note "how the capture was made"]

The name is the profile name of the launches (dslash_cg_f32 for one RHS, dslash_cg_f32_kK
for K), the variant the stencil variant the capture ran (EIG_DSLASH_VARIANT=N).
"""
import argparse
import csv
import hashlib
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STENCIL_SOURCES = ["dslash32.cuh", "dslash32.cu", "dslash32d_rb1.cu", "dslash32d_rb2.cu", "dslash32pp.cuh",
                   "dslash32p2.cu", "dslash32p3.cu", "dslash32p3f.cu"]


def stencil_sha1() -> str:
    h = hashlib.sha1()
    for f in STENCIL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_0707_0131_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def cg_algorithmic_bytes(sites: int, k: int, links: int) -> float:
    # CG pass 2 in FP32: links, then per RHS u read, r read and written
    return sites * (4 * (48 if links == 12 else 72) + k * 3 * 96)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("csv")
    ap.add_argument("--name", default="dslash_cg_f32_k16")
    ap.add_argument("--sites", type=int, required=True)
    ap.add_argument("--k", type=int, required=True)
    ap.add_argument("--links", type=int, default=12)
    ap.add_argument("--variant", type=int, required=True)
    ap.add_argument("--note", default="")
    a = ap.parse_args()
    per = {}
    with open(a.csv) as f:
        rows = [r for r in csv.reader(f) if len(r) > 5]
    hdr = rows[0]
    i_id, i_m, i_v = hdr.index("ID"), hdr.index("Metric Name"), hdr.index("Metric Value")
    unit_i = hdr.index("Metric Unit")
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    for r in rows[1:]:
        if r[i_m] in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            per.setdefault(r[i_id], 0.0)
            per[r[i_id]] += float(r[i_v].replace(",", "")) * scale.get(r[unit_i], 1)
    alg = cg_algorithmic_bytes(a.sites, a.k, a.links)
    # the same kernel may also run single-RHS products (the eigCG solves): keep the
    # launches whose traffic is that of a k-RHS product
    launches = [b for b in per.values() if b >= 0.5 * alg]
    if not launches:
        raise SystemExit("no captured launch moves the bytes of a %d-RHS product" % a.k)
    ratio = sum(launches) / len(launches) / alg
    out_path = os.path.join(ROOT, "configs", "traffic.json")
    data = json.load(open(out_path)) if os.path.exists(out_path) else {}
    entry = {"dram_over_algorithmic": ratio, "launches_captured": len(launches),
             "dram_bytes_per_launch": sum(launches) / len(launches), "algorithmic_bytes_per_launch": alg,
             "stencil_sha1": stencil_sha1(), "variant": a.variant, "link_reals": a.links, "capture": a.note}
    # one entry per (stencil sources, variant, link form); a new capture replaces the old one
    key = (entry["stencil_sha1"], a.variant, a.links)
    kept = [e for e in data.get(a.name, []) if (e["stencil_sha1"], e["variant"], e["link_reals"]) != key]
    data[a.name] = kept + [entry]
    json.dump(data, open(out_path, "w"), indent=1)
    print(json.dumps(entry, indent=1))


if __name__ == "__main__":
    main()
