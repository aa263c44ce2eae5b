import json
import os
import subprocess
import sys
import tempfile

from .. import build as _build

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    exe = os.path.join(tempfile.mkdtemp(), "alu_peak")
    subprocess.check_call([_build.nvcc()] + _build.ARCH + ["-O3", "-o", exe, os.path.join(HERE, "alu_peak.cu")])
    smi = subprocess.Popen(["nvidia-smi", "--query-gpu=clocks.sm,clocks.max.sm", "--format=csv,noheader,nounits",
                            "-lms", "50"], stdout=subprocess.PIPE, text=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    smi.terminate()
    clocks = [l.split(",") for l in smi.communicate()[0].splitlines() if "," in l]
    res = json.loads(out)
    res["sm_mhz_max_seen"] = max(float(c[0]) for c in clocks) if clocks else None
    sms = res["sms"]
    mhz = res["sm_mhz_max_seen"] or 2070.0
    for r in res["results"]:
        r["per_sm_per_clk"] = r["per_s"] / sms / (mhz * 1e6)
    print(json.dumps(res))


if __name__ == "__main__":
    sys.exit(main())
