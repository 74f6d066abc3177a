import json

from . import measure

print(json.dumps(measure(), indent=1))
