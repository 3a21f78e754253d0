"""Host logic of the bound-variant sweep tool (no GPU): argument checks and
the markdown tables it writes."""
import pytest

from paper_1806_05385_gb300 import sweep


def test_unknown_sweep_is_rejected_before_any_device_work():
    with pytest.raises(SystemExit) as e:
        sweep.main(["--sweeps", "bounds,nope"])
    assert e.value.code == 2
    with pytest.raises(SystemExit):
        sweep.main(["--sweeps", ""])


def test_markdown_tables():
    rows = [dict(sweep="bounds", mode="rolling", bound="zenon", ms=0.5, ste=0.25, pixels=10, hits=3),
            dict(sweep="bounds", mode="rolling", bound="trivial", ms=None, error="overflow"),
            dict(sweep="alpha", alpha=2.0, mode="foveated", ms=1.25, ste=0.5)]
    md = sweep.to_markdown(rows)
    lines = md.splitlines()
    # One table per sweep, in the tool's own order, without the raw counts.
    assert lines[0] == "### bounds" and "### alpha" in lines
    assert lines.index("### bounds") < lines.index("### alpha")
    head = lines[2]
    assert head == "| mode | bound | ms | ste | error |"
    assert "pixels" not in md and "hits" not in md
    # STE as a percentage, times with three decimals, missing cells empty,
    # a failed run's time as a dash.
    assert "| rolling | zenon | 0.500 | 25.0 % |  |" in lines
    assert "| rolling | trivial | - |  | overflow |" in lines
    assert "| 2.000 | foveated | 1.250 | 50.0 % |" in lines
